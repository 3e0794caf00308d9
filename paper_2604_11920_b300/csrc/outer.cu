// outer.cu -- the outer nonlinear loop of the inversion (the paragraph after
// Eq. 6 of the paper): solve Eq. 6 for the model perturbation, update the
// model, rebuild G from the updated model, and repeat until the RMS traveltime
// error falls below a threshold.  Every step runs in the library's kernels:
// the kernel table from the model and the value re-expansion (build_g.cu),
// the FP64 product G m, the residual and its sum of squares (here), the LSQR
// solve (lsqr.cu) and the model update (here).  The host only reads the RMS
// once per outer iteration to take the stopping decision.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pdst {

constexpr int OT = 256;         // threads per block
constexpr int OMAXBLK = 1024;   // blocks of the residual kernel

// r = d - y and one partial sum of r^2 per block (fixed order within the
// block: thread-strided, then warps in order).
__global__ void __launch_bounds__(OT) k_resid_ss(int64_t m, const double *__restrict__ d,
                                                 const double *__restrict__ y, double *r,
                                                 double *part) {
    __shared__ double red[OT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = d[i] - y[i];
        r[i] = v;
        s += v * v;
    }
    s = warp_sum(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < OT / 32; ++i) b += red[i];
        part[blockIdx.x] = b;
    }
}

// Sum of the block partials in block order (one thread).
__global__ void k_sum_parts(int nb, const double *__restrict__ part, double *out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    *out = s;
}

// m += dm.
__global__ void k_axpy1(int32_t n, const double *__restrict__ dm, double *mv) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        mv[j] = mv[j] + dm[j];
}

static unsigned blocks_for(int64_t work, int device) {
    int64_t b = (work + OT - 1) / OT;
    const int64_t cap = std::min<int64_t>((int64_t)num_sms(device) * 4, OMAXBLK);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

}  // namespace pdst

using namespace pdst;

extern "C" void pdst_outer_opts_default(pdst_outer_opts *o) {
    if (!o) return;
    *o = pdst_outer_opts{};
    o->max_outer = 8;
    o->rms_tol = 0.0;
    o->min_decrease = 0.01;
    o->z0_factor = 1.2;
    o->kernel_power = 1.0;
    pdst_lsqr_opts_default(&o->inner);
}

extern "C" pdst_status pdst_outer_loop(pdst_handle_t h, const double *d_obs_dev,
                                       const double *periods_host, double w, double lambda,
                                       int32_t itmax, double tol, const pdst_outer_opts *opts_in,
                                       double *m_out_dev, double *rms_hist_host,
                                       pdst_outer_info *info, void *stream) {
    PDST_CHECK_ARG(h != nullptr, "pdst_outer_loop: handle is NULL");
    PDST_CHECK_ARG(h->m == 0 || d_obs_dev, "pdst_outer_loop: d_obs is NULL");
    PDST_CHECK_ARG(periods_host && m_out_dev, "pdst_outer_loop: NULL pointer argument");
    pdst_outer_opts o;
    pdst_outer_opts_default(&o);
    if (opts_in) o = *opts_in;
    PDST_CHECK_ARG(o.max_outer >= 0 && o.max_outer <= 1000,
                   "pdst_outer_loop: max_outer must be in [0, 1000]");
    PDST_CHECK_ARG(std::isfinite(o.rms_tol) && o.rms_tol >= 0.0,
                   "pdst_outer_loop: rms_tol must be finite and >= 0");
    PDST_CHECK_ARG(std::isfinite(o.min_decrease) && o.min_decrease >= 0.0 && o.min_decrease < 1.0,
                   "pdst_outer_loop: min_decrease must be in [0, 1)");
    PDST_CHECK_ARG(h->m > 0, "pdst_outer_loop: G has no rows");
    if (!h->vals[PDST_F64].present) {
        set_error("pdst_outer_loop: the handle keeps no FP64 values (needed for the misfit)");
        return PDST_ERR_STATE;
    }
    if (!h->has_lengths) {
        set_error("pdst_outer_loop: the handle was built without keep_lengths");
        return PDST_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = h->m;
    const int32_t n = h->n;
    DevBuf K, y, r, dm, mprev, part, tot;
    PDST_TRY(K.alloc(sizeof(double) * (size_t)h->H * h->n_periods * h->nz));
    PDST_TRY(y.alloc(sizeof(double) * m));
    PDST_TRY(r.alloc(sizeof(double) * m));
    PDST_TRY(dm.alloc(sizeof(double) * std::max<int32_t>(n, 1)));
    PDST_TRY(mprev.alloc(sizeof(double) * std::max<int32_t>(n, 1)));
    PDST_TRY(part.alloc(sizeof(double) * OMAXBLK));
    PDST_TRY(tot.alloc(sizeof(double)));
    PDST_CUDA(cudaMemsetAsync(m_out_dev, 0, sizeof(double) * n, s));

    std::vector<double> hist;
    int updates = 0, reason = 0, inner_iters = 0;
    bool reverted = false;
    const unsigned nb = blocks_for(m, h->device);
    for (;;) {
        // G of the current model, its predicted data and the RMS misfit
        PDST_TRY(pdst_depth_kernels_from_model(h, periods_host, o.z0_factor, o.kernel_power,
                                               m_out_dev, K.as<double>(), stream));
        PDST_TRY(pdst_set_depth_kernels(h, K.as<double>(), stream));
        PDST_TRY(pdst_apply_G(h, PDST_F64, 0, m_out_dev, y.as<double>(), stream));
        k_resid_ss<<<nb, OT, 0, s>>>(m, d_obs_dev, y.as<double>(), r.as<double>(),
                                     part.as<double>());
        k_sum_parts<<<1, 32, 0, s>>>((int)nb, part.as<double>(), tot.as<double>());
        PDST_CUDA(cudaGetLastError());
        double ss = 0.0;
        PDST_CUDA(cudaMemcpyAsync(&ss, tot.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        PDST_CUDA(cudaStreamSynchronize(s));
        const double rms = std::sqrt(ss / (double)m);
        if (!std::isfinite(rms)) {
            set_error("pdst_outer_loop: non-finite RMS misfit after %d updates", updates);
            return PDST_ERR_BREAKDOWN;
        }
        hist.push_back(rms);
        if (rms <= o.rms_tol) {
            reason = 1;
            break;
        }
        if (hist.size() > 1 && rms > (1.0 - o.min_decrease) * hist[hist.size() - 2]) {
            reason = 2;
            if (rms > hist[hist.size() - 2]) {   // keep the model with the smaller misfit
                PDST_CUDA(cudaMemcpyAsync(m_out_dev, mprev.p, sizeof(double) * n,
                                          cudaMemcpyDeviceToDevice, s));
                reverted = true;
            }
            break;
        }
        if (updates == o.max_outer) {
            reason = 3;
            break;
        }
        // Eq. 6 for the update, on G of the current model
        if (o.inner.precond == 1)
            PDST_TRY(pdst_set_col_scaling(h, nullptr, w, lambda, stream));
        else if (o.inner.precond == 2)
            PDST_TRY(pdst_set_block_precond(h, nullptr, w, lambda, stream));
        pdst_lsqr_info li{};
        PDST_TRY(pdst_lsqr(h, r.as<double>(), w, lambda, itmax, tol, dm.as<double>(), &li,
                           &o.inner, stream));
        inner_iters += li.iters;
        PDST_CUDA(cudaMemcpyAsync(mprev.p, m_out_dev, sizeof(double) * n,
                                  cudaMemcpyDeviceToDevice, s));
        k_axpy1<<<blocks_for(n, h->device), OT, 0, s>>>(n, dm.as<double>(), m_out_dev);
        PDST_CUDA(cudaGetLastError());
        ++updates;
    }
    PDST_CUDA(cudaStreamSynchronize(s));
    if (rms_hist_host)
        for (size_t i = 0; i < hist.size(); ++i) rms_hist_host[i] = hist[i];
    if (info) {
        *info = pdst_outer_info{};
        info->updates = updates;
        info->reason = reason;
        info->inner_iters = inner_iters;
        info->rms_first = hist.front();
        info->rms_final = reverted ? hist[hist.size() - 2] : hist.back();
    }
    return PDST_OK;
}
