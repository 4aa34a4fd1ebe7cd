// model.cu -- a fitted kernel ridge regression model kept ready for
// prediction (arXiv 2111.10140, Sec. 4.3: K(Z, X) alpha ~ sum_l eta_l
// Phi_{Z,l} D_l Phi_{X,l}^* alpha).
//
// For fixed coefficients alpha the factor h_l = D_l Phi_{X,l}^* alpha -- the
// spread of alpha onto window l's oversampled grid, convolved with the
// kernel's Fourier multiplier -- is the same for every set of test points.
// The model computes it once per window and keeps the real grids; a
// prediction then only bins its test points and gathers from those grids,
// with the spread, FFT and gather kernels of krr_predict in its precision.
//
// Test points outside the plan's ball cannot use grids of the plan's frame.
// The model therefore keeps, where the bandwidth allows it, a second grid per
// window in a wider frame: same centre, scale divided by rho in (1, 2], so
// every point within rho times the nodes' radius maps into the ball.  The
// frame shrinks the kernel's width on the torus by rho; rho is the largest
// value (at most 2) for which the Gaussian's Fourier transform at the band
// edge, exp(-(pi ell_l n / (2 rho))^2), stays below 1e-12, so the wider frame
// costs no accuracy at the plan's n.  A window whose test points reach even
// beyond that is summed as krr_predict sums it (joint frame of nodes and test
// points, the plan's own grid), one such window per model at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"

struct krr_model {
    anova_plan* plan = nullptr;
    double* alpha = nullptr;          // device copy of the coefficients (N)
    void* grids = nullptr;            // device, per window the plan-frame grid and the wide-frame grid
    std::vector<size_t> off, off_wide;
    std::vector<anova::WindowPlan> wide;   // wide-frame parameters (dA == 0: no wide grid)
    size_t elems = 0;
    bool fp64 = true;                 // grids and gathers in FP64 (else FP32), as krr_predict
    std::mutex fallback;              // serialises windows summed on the plan's own grids
};

namespace anova {

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_model_sum(const T* __restrict__ tmp, const double* __restrict__ eta, int P, int64_t M, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < P; l++) acc += eta[l] * (double)tmp[l * M + i];
        out[i] = acc;
    }
}

// rho of the wide frame for window l (1 when no widening is possible)
static double wide_rho(const WindowPlan& w) {
    const double pi = 3.14159265358979323846;
    const double rho = pi * w.ell_l * w.n / (2.0 * std::sqrt(std::log(1e12)));
    return std::min(2.0, rho);
}

template <typename T>
static anova_status convolved_grid(anova_plan* plan, const WindowPlan& w, const double* alpha, T* grid,
                                   cudaStream_t st) {
    size_t ge = 1;
    for (int t = 0; t < w.dA; t++) ge *= w.nos;
    ANOVA_CUDA_TRY(cudaMemsetAsync(grid, 0, ge * sizeof(T), st));
    if (plan->N == 0) return ANOVA_OK;
    ANOVA_TRY(spread_window<T>(plan, w, w.X, alpha, 1, grid, st));
    return fft_convolve_window<T>(plan, w, grid, st);
}

template <typename T>
static anova_status model_grids(krr_model* md, cudaStream_t st) {
    anova_plan* plan = md->plan;
    T* g = static_cast<T*>(md->grids);
    for (int l = 0; l < plan->P; l++) {
        ANOVA_TRY(convolved_grid<T>(plan, plan->win[l], md->alpha, g + md->off[l], st));
        if (md->wide[l].dA == 0) continue;
        WindowPlan wide;
        anova_status s = window_widened(plan, l, wide_rho(plan->win[l]), wide, st);
        if (s == ANOVA_OK) s = convolved_grid<T>(plan, wide, md->alpha, g + md->off_wide[l], st);
        if (s == ANOVA_OK && cudaStreamSynchronize(st) != cudaSuccess) s = ANOVA_ECUDA;
        WindowPlan keep = wide;       // frame and binning parameters only
        keep.X = PointSet();
        keep.wtab = nullptr;
        keep.wtap64 = nullptr;
        keep.D64 = nullptr;
        keep.D32 = nullptr;
        keep.tw64 = nullptr;
        keep.tw32 = nullptr;
        keep.xw = nullptr;
        window_release_reframed(wide);
        if (s != ANOVA_OK) return s;
        md->wide[l] = keep;
    }
    return ANOVA_OK;
}

// window l at test coordinates zl: gather from the plan-frame grid, else
// from the wide-frame grid, else the full per-window summation
template <typename T>
static anova_status model_window(krr_model* md, int l, const double* zl, int64_t M, T* out, cudaStream_t st) {
    anova_plan* plan = md->plan;
    const WindowPlan& w = plan->win[l];
    const double RB = 0.25 - 0.5 * plan->epsB;
    double rmax = 0.0;
    ANOVA_TRY(max_radius(plan, zl, M, w.dA, w.centre, &rmax, st));
    const T* g = static_cast<const T*>(md->grids);
    const WindowPlan* fw = nullptr;
    const T* grid = nullptr;
    if (w.scale * rmax <= RB) {
        fw = &w;
        grid = g + md->off[l];
    } else if (md->wide[l].dA != 0 && md->wide[l].scale * rmax <= RB) {
        fw = &md->wide[l];
        grid = g + md->off_wide[l];
    }
    if (!fw) {
        std::lock_guard<std::mutex> lock(md->fallback);
        return predict_window<T>(plan, l, md->alpha, zl, M, out, st);
    }
    if (plan->N == 0) {
        ANOVA_CUDA_TRY(cudaMemsetAsync(out, 0, M * sizeof(T), st));
        return ANOVA_OK;
    }
    WindowPlan wz = *fw;   // binning parameters of the frame
    PointSet zs;
    anova_status s = build_pointset(plan, wz, zl, M, fw->dA, fw->centre, fw->scale, zs, st);
    if (s == ANOVA_OK) s = gather_window<T>(plan, *fw, zs, grid, out, st);
    free_pointset_async(zs, st);
    wz.X = PointSet();
    return s;
}

template <typename T>
static anova_status model_predict(krr_model* md, const double* Z, int64_t M, int64_t ldz, double* out,
                                  cudaStream_t st) {
    anova_plan* plan = md->plan;
    const int P = plan->P;
    T* tmp = nullptr;
    double* zw = nullptr;
    Scratch scratch(st);
    ANOVA_CUDA_TRY(scratch.alloc(&tmp, (size_t)M * P * sizeof(T)));
    ANOVA_CUDA_TRY(scratch.alloc(&zw, (size_t)M * 3 * sizeof(double)));
    anova_status s = ANOVA_OK;
    for (int l = 0; l < P && s == ANOVA_OK; l++) {
        s = extract_window(plan, Z, M, ldz, plan->win[l], zw, st);
        if (s == ANOVA_OK) s = model_window<T>(md, l, zw, M, tmp + (int64_t)l * M, st);
    }
    if (s == ANOVA_OK) {
        k_model_sum<T><<<grid_for(M, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(tmp, plan->eta_dev, P, M,
                                                                                      out);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("krr_model_predict: ") + cudaGetErrorString(e));
            s = ANOVA_ECUDA;
        }
    }
    return s;
}

}  // namespace anova

using namespace anova;

extern "C" {

anova_status krr_model_create(anova_plan* plan, const double* alpha, void* stream, krr_model** out) {
    if (!plan || !out || (plan->N > 0 && !alpha)) {
        set_error("krr_model_create: bad plan, alpha or output pointer");
        return ANOVA_EINVAL;
    }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    krr_model* md = new (std::nothrow) krr_model();
    if (!md) return ANOVA_ENOMEM;
    md->plan = plan;
    md->fp64 = (plan->precision & ANOVA_FP64) != 0;
    const size_t esz = md->fp64 ? sizeof(double) : sizeof(float);
    md->off.resize(plan->P);
    md->off_wide.resize(plan->P);
    md->wide.resize(plan->P);
    for (int l = 0; l < plan->P; l++) {
        size_t ge = 1;
        for (int t = 0; t < plan->win[l].dA; t++) ge *= plan->win[l].nos;
        ge = (ge + 63) & ~(size_t)63;           // 256-byte aligned window grids
        md->off[l] = md->elems;
        md->elems += ge;
        if (plan->N > 0 && wide_rho(plan->win[l]) > 1.05) {
            md->wide[l].dA = plan->win[l].dA;   // marks a wide grid, filled by model_grids
            md->off_wide[l] = md->elems;
            md->elems += ge;
        }
    }
    anova_status s = ANOVA_OK;
    if (anova::dev_malloc((void**)&md->alpha, std::max<int64_t>(plan->N, 1) * sizeof(double)) != cudaSuccess ||
        anova::dev_malloc((void**)&md->grids, std::max<size_t>(md->elems, 1) * esz) != cudaSuccess) {
        set_error("krr_model_create: out of device memory");
        s = ANOVA_ENOMEM;
    }
    if (s == ANOVA_OK && plan->N > 0 &&
        cudaMemcpyAsync(md->alpha, alpha, plan->N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        set_error("krr_model_create: copy of alpha failed");
        s = ANOVA_ECUDA;
    }
    if (s == ANOVA_OK) s = md->fp64 ? model_grids<double>(md, st) : model_grids<float>(md, st);
    if (s == ANOVA_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("krr_model_create: ") + cudaGetErrorString(e));
            s = ANOVA_ECUDA;
        }
    }
    if (s != ANOVA_OK) {
        cudaFree(md->alpha);
        cudaFree(md->grids);
        delete md;
        return s;
    }
    *out = md;
    return ANOVA_OK;
}

anova_status krr_model_predict(krr_model* md, const double* Z, int64_t M, int64_t ldz, double* out, void* stream) {
    if (!md || M < 0 || ldz < md->plan->d || (M > 0 && (!Z || !out))) {
        set_error("krr_model_predict: bad model, sizes or pointers");
        return ANOVA_EINVAL;
    }
    if (M == 0) return ANOVA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t w0 = wait_timeouts_on(st);
    const anova_status s =
        md->fp64 ? model_predict<double>(md, Z, M, ldz, out, st) : model_predict<float>(md, Z, M, ldz, out, st);
    return waits_moved(w0, st, "krr_model_predict", s);
}

void krr_model_destroy(krr_model* md) {
    if (!md) return;
    cudaFree(md->alpha);
    cudaFree(md->grids);
    delete md;
}

}  // extern "C"

extern "C" anova_status krr_model_alpha(const krr_model* model, double* out, void* stream) {
    if (!model || (model->plan && model->plan->N > 0 && !out)) {
        anova::set_error("krr_model_alpha: NULL model or output");
        return ANOVA_EINVAL;
    }
    const int64_t N = model->plan ? model->plan->N : 0;
    if (N == 0) return ANOVA_OK;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(out, model->alpha, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                   (cudaStream_t)stream));
    return ANOVA_OK;
}
