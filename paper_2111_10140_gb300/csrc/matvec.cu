// matvec.cu -- the ANOVA matrix-vector product, CG for kernel ridge regression
// and prediction (arXiv 2111.10140):
//
//   K alpha = sum_l eta_l K_l alpha ~= sum_l eta_l Phi_l D_l Phi_l^* alpha
//       (Sec. 4.3, Sec. 5: P fast summations, one per window, weighted sum)
//   (K + lambda I) alpha = y by conjugate gradients (Sec. 2, Hestenes-Stiefel)
//   s = sum_l eta_l Phi_{z,l} D_l Phi_l^* alpha at test points (Sec. 4.3)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace anova {

// --------------------------------------------------------------- stage clock
void clock_begin(anova_plan* plan, int stage, cudaStream_t st) {
    StageClock& c = plan->clock;
    if (!c.enabled) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    c.open[stage] = (int)c.ev.size();
    c.ev.push_back(a);
    c.ev.push_back(b);
    c.stage_of_pair.push_back(stage);
}

// closes the stage's most recent open pair (stages may nest: 4 inside 0, 5 inside 2)
void clock_end(anova_plan* plan, int stage, int launches, cudaStream_t st) {
    StageClock& c = plan->clock;
    if (!c.enabled || c.open[stage] < 0) return;
    cudaEventRecord(c.ev[c.open[stage] + 1], st);
    c.open[stage] = -1;
    c.launches[stage] += launches;
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// deterministic block sum (blockDim.x == kThreads); result valid in all threads
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

// sum of nblk partials in a fixed order, inside every block
__device__ double sum_partials(const double* __restrict__ part, int nblk, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += part[i];
    return block_sum(v, sh);
}

// ------------------------------------------------------------ window sum
// out_i = sum_l eta_l tmp_l[i]
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads)
k_window_sum(const Tin* __restrict__ tmp, const double* __restrict__ eta, int P, int64_t N,
             Tout* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < P; l++) acc += eta[l] * (double)tmp[l * N + i];
        out[i] = (Tout)acc;
    }
}

// FP32 operator: out_i = sum_l eta_l tmp_l[i] in FP32 (the weights rounded to
// FP32 once per thread), four elements per step when `vec` (N a multiple of 4,
// tmp and out 16-byte aligned).
// The FP64 form above converts every term to FP64, which on this GPU's FP64
// rate costs more than the memory traffic.
__global__ void __launch_bounds__(kThreads)
k_window_sum_f32(const float* __restrict__ tmp, const double* __restrict__ eta, int P, int64_t N,
                 float* __restrict__ out, int vec) {
    __shared__ float e[64];
    for (int l = threadIdx.x; l < 64; l += blockDim.x) e[l] = l < P ? (float)eta[l] : 0.f;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (vec && P <= 64) {
        const int64_t N4 = N >> 2;
        for (int64_t i = t0; i < N4; i += stride) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int l = 0; l < P; l++) {
                const float4 v = reinterpret_cast<const float4*>(tmp + (int64_t)l * N)[i];
                acc.x = fmaf(e[l], v.x, acc.x);
                acc.y = fmaf(e[l], v.y, acc.y);
                acc.z = fmaf(e[l], v.z, acc.z);
                acc.w = fmaf(e[l], v.w, acc.w);
            }
            reinterpret_cast<float4*>(out)[i] = acc;
        }
        return;
    }
    for (int64_t i = t0; i < N; i += stride) {
        float acc = 0.f;
        for (int l = 0; l < P; l++) acc = fmaf(l < 64 ? e[l] : (float)eta[l], tmp[(int64_t)l * N + i], acc);
        out[i] = acc;
    }
}

// -------------------------------------------------------------- matvec core
// The FP32 product with the 1-D / 2-D windows' chain (spread, box FFT, gather)
// on the plan's second stream beside the 3-D windows' chain: the two touch
// disjoint grids and result slices, and the 1-D / 2-D box FFT (one block per
// window) or the 3-D FFT then run while the other chain keeps the SMs busy.
// A fork / join by events, so a graph captured on `st` holds both branches.
static bool overlap_ok(const anova_plan* plan) {
    if ((plan->overlap12 & 3) == 0 || plan->clock.enabled || !plan->side || !plan->side_hi ||
        plan->dense_windows.empty())
        return false;
    bool has12 = false, has3 = false;
    for (const auto& g : plan->dense_groups) (g[0] / 100 < 3 ? has12 : has3) = true;
    if (!has12 || !has3) return false;
    for (int l = 0; l < plan->P; l++) {
        const WindowPlan& w = plan->win[l];
        if (w.dense && w.dA < 3 && !w.fft12) return false;   // its FFT would run on the other stream
    }
    return true;
}

template <typename T>
static anova_status windows_apply_overlapped(anova_plan* plan, const void* alpha, int alpha_is_double, T* tmp,
                                             cudaStream_t st) {
    const int64_t N = plan->N;
    const int when = plan->overlap12 & 3;
    cudaStream_t side = (plan->overlap12 & 4) ? plan->side_hi : plan->side;
    ANOVA_CUDA_TRY(cudaMemsetAsync(plan->grid, 0, plan->grid_elems * sizeof(T), st));
    ANOVA_TRY(dense3_spread_all<T>(plan, alpha, alpha_is_double, st, nullptr, kDenseSort));
    anova_status s3 = ANOVA_OK;
    if (when == 3) s3 = dense3_spread_all<T>(plan, alpha, alpha_is_double, st, nullptr, kDense3);
    ANOVA_CUDA_TRY(cudaEventRecord(plan->ev_fork, st));
    if (when == 2 && s3 == ANOVA_OK) s3 = dense3_spread_all<T>(plan, alpha, alpha_is_double, st, nullptr, kDense3);
    // the fork is waited on and the join recorded whatever happened, so a capture on `st` stays well formed
    const cudaError_t ef = cudaStreamWaitEvent(side, plan->ev_fork, 0);
    anova_status s12 = ef == cudaSuccess ? ANOVA_OK : ANOVA_ECUDA;
    if (s12 == ANOVA_OK) s12 = dense3_spread_all<T>(plan, alpha, alpha_is_double, side, nullptr, kDense12);
    if (s12 == ANOVA_OK) s12 = fft12_box_all<T>(plan, side);
    if (s12 == ANOVA_OK) s12 = dense3_gather_all<T>(plan, side, kDense12);
    const cudaError_t ej = cudaEventRecord(plan->ev_join, side);
    if (when == 1 && s3 == ANOVA_OK) s3 = dense3_spread_all<T>(plan, alpha, alpha_is_double, st, nullptr, kDense3);
    for (int l = 0; l < plan->P && s3 == ANOVA_OK; l++) {
        const WindowPlan& w = plan->win[l];
        if (!w.dense) s3 = spread_window<T>(plan, w, w.X, alpha, alpha_is_double, grid_of<T>(plan, w), st);
    }
    if (s3 == ANOVA_OK && !plan->fft3_windows.empty()) s3 = fft3_box_all<T>(plan, st);
    for (int l = 0; l < plan->P && s3 == ANOVA_OK; l++) {
        const WindowPlan& w = plan->win[l];
        if (fft3_box_supported(w) || w.fft12) continue;
        s3 = fft_convolve_window<T>(plan, w, grid_of<T>(plan, w), st);
    }
    if (s3 == ANOVA_OK) s3 = dense3_gather_all<T>(plan, st, kDense3);
    for (int l = 0; l < plan->P && s3 == ANOVA_OK; l++) {
        const WindowPlan& w = plan->win[l];
        if (!w.dense) s3 = gather_window<T>(plan, w, w.X, grid_of<T>(plan, w), tmp + (int64_t)l * N, st);
    }
    const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(st, plan->ev_join, 0) : ej;
    if (ef != cudaSuccess) {
        set_error(std::string("anova product: forking the 1-D / 2-D stream: ") + cudaGetErrorString(ef));
        return ANOVA_ECUDA;
    }
    if (s12 != ANOVA_OK) return s12;
    if (s3 != ANOVA_OK) return s3;
    if (ew != cudaSuccess) {
        set_error(std::string("anova product: joining the 1-D / 2-D stream: ") + cudaGetErrorString(ew));
        return ANOVA_ECUDA;
    }
    return ANOVA_OK;
}

// tmp_l = K_l alpha for every window (fast summation of Sec. 4.2 Eq. fastsum).
// `tmp` must be plan->tmp: the batched dense kernels write their slices of it.
template <typename T>
static anova_status windows_apply(anova_plan* plan, const void* alpha, int alpha_is_double, T* tmp,
                                  cudaStream_t st) {
    if constexpr (sizeof(T) == 4)
        if (overlap_ok(plan)) return windows_apply_overlapped<T>(plan, alpha, alpha_is_double, tmp, st);
    const int64_t N = plan->N;
    ANOVA_CUDA_TRY(cudaMemsetAsync(plan->grid, 0, plan->grid_elems * sizeof(T), st));
    int nl = 0;
    clock_begin(plan, 0, st);
    if (!plan->dense_windows.empty()) {
        ANOVA_TRY(dense3_spread_all<T>(plan, alpha, alpha_is_double, st, &nl));
    }
    // windows not on the batched dense kernels: generic kernels, one window at a time
    // (FP64 runs the dense 1-D / 2-D windows here too)
    auto generic = [&](const WindowPlan& w) { return !w.dense || (sizeof(T) == 8 && w.dA < 3); };
    for (int l = 0; l < plan->P; l++) {
        const WindowPlan& w = plan->win[l];
        if (!generic(w)) continue;
        ANOVA_TRY(spread_window<T>(plan, w, w.X, alpha, alpha_is_double, grid_of<T>(plan, w), st));
        nl++;
    }
    clock_end(plan, 0, nl, st);
    nl = 0;
    clock_begin(plan, 1, st);
    if (!plan->fft3_windows.empty()) {
        ANOVA_TRY(fft3_box_all<T>(plan, st));
        nl += plan->fft3_slab ? 3 : 5;
    }
    if (!plan->fft12_windows.empty()) {
        ANOVA_TRY(fft12_box_all<T>(plan, st));
        nl++;
    }
    for (int l = 0; l < plan->P; l++) {
        const WindowPlan& w = plan->win[l];
        if (fft3_box_supported(w) || w.fft12) continue;
        ANOVA_TRY(fft_convolve_window<T>(plan, w, grid_of<T>(plan, w), st));
        nl += 2 * w.dA;
    }
    clock_end(plan, 1, nl, st);
    nl = 0;
    clock_begin(plan, 2, st);
    if (!plan->dense_windows.empty()) {
        ANOVA_TRY(dense3_gather_all<T>(plan, st));
        nl += (int)plan->dense_groups.size();
    }
    for (int l = 0; l < plan->P; l++) {
        const WindowPlan& w = plan->win[l];
        if (!generic(w)) continue;
        ANOVA_TRY(gather_window<T>(plan, w, w.X, grid_of<T>(plan, w), tmp + (int64_t)l * N, st));
        nl++;
    }
    clock_end(plan, 2, nl, st);
    return ANOVA_OK;
}

static bool has_precision(const anova_plan* plan, int dtype) {
    return (dtype == ANOVA_FP64 || dtype == ANOVA_FP32) && (plan->precision & dtype);
}

template <typename T>
static anova_status matvec_one(anova_plan* plan, const T* alpha, T* out, cudaStream_t st) {
    const int64_t N = plan->N;
    if (N == 0) return ANOVA_OK;
    T* tmp = static_cast<T*>(plan->tmp);
    ANOVA_TRY(windows_apply<T>(plan, alpha, sizeof(T) == 8, tmp, st));
    clock_begin(plan, 3, st);
    if constexpr (sizeof(T) == 4)
        k_window_sum_f32<<<grid_for((N + 3) / 4, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            tmp, plan->eta_dev, plan->P, N, out,
            (N % 4 == 0 && reinterpret_cast<uintptr_t>(tmp) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0)
                ? 1 : 0);
    else
        k_window_sum<T, T><<<grid_for(N, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            tmp, plan->eta_dev, plan->P, N, out);
    ANOVA_CHECK_LAUNCH();
    clock_end(plan, 3, 1, st);
    return ANOVA_OK;
}

// ================================================================== CG
// Vectors (FP64): r, p, q, x stored in plan->cg_vec; scalars in cg_scal:
//   [0] yy, [1] result scratch, [2 ...] rr history (one entry per iteration)
__global__ void __launch_bounds__(kThreads)
k_cg_init(const double* __restrict__ b, int64_t N, double* __restrict__ x, double* __restrict__ r,
          double* __restrict__ p, int zero_x, double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i];
        if (zero_x) x[i] = 0.0;
        r[i] = v;
        p[i] = v;
        acc += v * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_reduce_to(const double* __restrict__ part, int nblk, double* __restrict__ dst) {
    __shared__ double sh[32];
    double v = sum_partials(part, nblk, sh);
    if (threadIdx.x == 0) *dst = v;
}

// q = sum_l eta_l tmp_l + lambda p; partial sums of p.q
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cg_q(const T* __restrict__ tmp, const double* __restrict__ eta, int P, int64_t N, double lambda,
       const double* __restrict__ p, double* __restrict__ q, double* __restrict__ part) {
    __shared__ double sh[32];
    __shared__ float ef[64];          // FP32 operator: the window sum in FP32 (one FP64 conversion per element)
    if (sizeof(T) == 4) {
        for (int l = threadIdx.x; l < 64; l += blockDim.x) ef[l] = l < P ? (float)eta[l] : 0.f;
        __syncthreads();
    }
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = lambda * p[i];
        if (sizeof(T) == 4 && P <= 64) {
            float s = 0.f;
            for (int l = 0; l < P; l++) s = fmaf(ef[l], (float)tmp[l * N + i], s);
            v += (double)s;
        } else {
            for (int l = 0; l < P; l++) v += eta[l] * (double)tmp[l * N + i];
        }
        q[i] = v;
        acc += p[i] * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// a = rr / (p.q); x += a p; r -= a q; partial sums of r.r
__global__ void __launch_bounds__(kThreads)
k_cg_update(const double* __restrict__ part_pq, int nblk, const double* __restrict__ rr_now, int64_t N,
            double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
            const double* __restrict__ q, double* __restrict__ part_rr) {
    __shared__ double sh[32];
    const double pq = sum_partials(part_pq, nblk, sh);
    const double a = *rr_now / pq;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = acc;
}

// b = rr_new / rr; p = r + b p; rr_next = rr_new
__global__ void __launch_bounds__(kThreads)
k_cg_pupdate(const double* __restrict__ part_rr, int nblk, const double* __restrict__ rr_now,
             double* __restrict__ rr_next, int64_t N, const double* __restrict__ r, double* __restrict__ p) {
    __shared__ double sh[32];
    const double rr_new = sum_partials(part_rr, nblk, sh);
    const double beta = rr_new / *rr_now;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *rr_next = rr_new;
}

// r = b - q (q already holds (K + lambda I) x); partial sums of r.r
__global__ void __launch_bounds__(kThreads)
k_residual(const double* __restrict__ b, const double* __restrict__ q, int64_t N, double* __restrict__ r,
           double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i] - q[i];
        r[i] = v;
        acc += v * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_axpy(int64_t N, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

struct CgBuffers {
    double *r, *p, *q, *x2, *scal, *part, *part2;
    int nblk;
};

static anova_status cg_buffers(anova_plan* plan, int maxit, CgBuffers& B) {
    const int64_t N = plan->N;
    const int nblk = grid_for(N, kThreads, 2 * plan->sm_count);
    if (!plan->cg_vec) ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->cg_vec, 4 * std::max<int64_t>(N, 1) * sizeof(double)));
    if (!plan->cg_part) ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->cg_part, 2 * 2 * plan->sm_count * sizeof(double)));
    if (plan->cg_hist < maxit + 8) {
        cudaFree(plan->cg_scal);
        plan->cg_scal = nullptr;
        plan->cg_hist = maxit + 8;
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->cg_scal, (plan->cg_hist + 4) * sizeof(double)));
    }
    B.r = plan->cg_vec;
    B.p = plan->cg_vec + N;
    B.q = plan->cg_vec + 2 * N;
    B.x2 = plan->cg_vec + 3 * N;
    B.scal = plan->cg_scal;
    B.part = plan->cg_part;
    B.part2 = plan->cg_part + 2 * plan->sm_count;
    B.nblk = nblk;
    return ANOVA_OK;
}

// Replay a captured launch sequence keyed by (kind, dtype, input, output,
// lambda): the first call with a key runs `launch` directly (so that one-time
// kernel attributes are set outside any capture), the second captures it into
// a CUDA graph, later calls replay that graph.  At most 16 graphs per plan.
template <typename F>
static anova_status run_cached(anova_plan* plan, int kind, int dtype, const void* in, void* out, double lambda,
                               cudaStream_t st, F&& launch) {
    if (!plan->use_graphs || plan->clock.enabled) return launch(st);
    for (auto& g : plan->graphs) {
        if (g.kind != kind || g.dtype != dtype || g.alpha != in || g.out != out || g.lambda != lambda) continue;
        if (g.exec) {
            ANOVA_CUDA_TRY(cudaGraphLaunch(g.exec, st));
            return ANOVA_OK;
        }
        if (!plan->capture_stream)
            ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        ANOVA_CUDA_TRY(cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal));
        anova_status cs = launch(plan->capture_stream);
        cudaError_t ce = cudaStreamEndCapture(plan->capture_stream, &graph);
        if (cs != ANOVA_OK) {
            if (graph) cudaGraphDestroy(graph);
            return cs;
        }
        if (ce != cudaSuccess) {
            set_error(std::string("graph capture: ") + cudaGetErrorString(ce));
            return ANOVA_ECUDA;
        }
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            set_error(std::string("graph instantiate: ") + cudaGetErrorString(ce));
            return ANOVA_ECUDA;
        }
        g.exec = exec;
        ANOVA_CUDA_TRY(cudaGraphLaunch(g.exec, st));
        return ANOVA_OK;
    }
    if (plan->graphs.size() >= 16) {
        if (plan->graphs.front().exec) cudaGraphExecDestroy(plan->graphs.front().exec);
        plan->graphs.erase(plan->graphs.begin());
    }
    plan->graphs.push_back({kind, dtype, in, out, lambda, nullptr});
    return launch(st);
}

// q = (K + lambda I) v with the operator of precision T; partial sums of v.q in B.part
template <typename T>
static anova_status apply_shifted(anova_plan* plan, double lambda, const double* v, double* q,
                                  const CgBuffers& B, cudaStream_t st) {
    T* tmp = static_cast<T*>(plan->tmp);
    return run_cached(plan, 1, (int)sizeof(T), v, q, lambda, st, [&](cudaStream_t s) -> anova_status {
        ANOVA_TRY(windows_apply<T>(plan, v, 1, tmp, s));
        clock_begin(plan, 3, s);
        k_cg_q<T><<<B.nblk, kThreads, 0, s>>>(tmp, plan->eta_dev, plan->P, plan->N, lambda, v, q, B.part);
        ANOVA_CHECK_LAUNCH();
        clock_end(plan, 3, 1, s);
        return ANOVA_OK;
    });
}

static anova_status read_scalar(const double* d, double* h, cudaStream_t st) {
    ANOVA_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// Plain CG on (K_T + lambda I) x = b, x_0 = 0 (FP64 vectors and scalars).
// Stops when ||r|| <= tol * ||b|| (checked every kCheckEvery iterations, which
// are queued without a host round trip in between), after maxit iterations, or
// -- when `stagnation` is set -- when the best residual of the last
// kStallWindow iterations is not below half the best one before them.
constexpr int kCheckEvery = 4;
constexpr int kStallWindow = 64;
template <typename T>
static anova_status cg_run(anova_plan* plan, double lambda, const double* b, double* x, double tol, int maxit,
                           const CgBuffers& B, int* iters, double* bb_out, cudaStream_t st, bool stagnation = false) {
    const int64_t N = plan->N;
    double* hist = B.scal + 2;
    k_cg_init<<<B.nblk, kThreads, 0, st>>>(b, N, x, B.r, B.p, 1, B.part);
    k_reduce_to<<<1, kThreads, 0, st>>>(B.part, B.nblk, hist);
    ANOVA_CHECK_LAUNCH();
    double bb = 0.0;
    ANOVA_TRY(read_scalar(hist, &bb, st));
    if (bb_out) *bb_out = bb;
    int it = 0;
    double rr = bb;
    double best = bb, best_at_window = bb;
    int window_start = 0;
    std::vector<double> hbuf(kCheckEvery);
    while (it < maxit && rr > tol * tol * bb && bb > 0.0) {
        const int batch = std::min(kCheckEvery, maxit - it);
        for (int k = 0; k < batch; k++) {
            ANOVA_TRY(apply_shifted<T>(plan, lambda, B.p, B.q, B, st));
            clock_begin(plan, 3, st);
            k_cg_update<<<B.nblk, kThreads, 0, st>>>(B.part, B.nblk, hist + it, N, x, B.r, B.p, B.q, B.part2);
            k_cg_pupdate<<<B.nblk, kThreads, 0, st>>>(B.part2, B.nblk, hist + it, hist + it + 1, N, B.r, B.p);
            ANOVA_CHECK_LAUNCH();
            clock_end(plan, 3, 2, st);
            it++;
        }
        ANOVA_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), hist + it - batch + 1, batch * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        for (int k = 0; k < batch; k++) {
            if (!std::isfinite(hbuf[k])) {
                set_error("CG residual is not finite");
                *iters = it;
                return ANOVA_ERANGE;
            }
            best = std::min(best, hbuf[k]);
        }
        rr = hbuf[batch - 1];
        if (stagnation && it - window_start >= kStallWindow) {
            if (best > 0.25 * best_at_window) break;    // residual norm not halved over the window
            best_at_window = best;
            window_start = it;
        }
    }
    *iters = it;
    return ANOVA_OK;
}

// true relative residual ||b - (K_T + lambda I) x|| / ||b||
template <typename T>
static anova_status true_residual(anova_plan* plan, double lambda, const double* b, const double* x,
                                  double bb, const CgBuffers& B, double* relres, cudaStream_t st) {
    ANOVA_TRY(apply_shifted<T>(plan, lambda, x, B.q, B, st));
    k_residual<<<B.nblk, kThreads, 0, st>>>(b, B.q, plan->N, B.r, B.part);
    k_reduce_to<<<1, kThreads, 0, st>>>(B.part, B.nblk, B.scal + 1);
    ANOVA_CHECK_LAUNCH();
    double rr = 0.0;
    ANOVA_TRY(read_scalar(B.scal + 1, &rr, st));
    *relres = (bb > 0.0) ? std::sqrt(rr / bb) : 0.0;
    return ANOVA_OK;
}

// Plain FP64 CG on (K64 + lambda I) x = b from x = 0, whatever the plan's
// precision (the plan must hold FP64 data): the fallback of the batched
// refined solver for systems whose FP32 corrections stop helping.
anova_status cg_fp64_solve(anova_plan* plan, double lambda, const double* b, double* x, double tol, int maxit,
                           int* iters, double* relres, cudaStream_t st) {
    *iters = 0;
    *relres = 0.0;
    if (plan->N == 0 || maxit < 1) return ANOVA_OK;
    CgBuffers B;
    ANOVA_TRY(cg_buffers(plan, maxit, B));
    double bb = 0.0;
    ANOVA_TRY(cg_run<double>(plan, lambda, b, x, tol, maxit, B, iters, &bb, st));
    return true_residual<double>(plan, lambda, b, x, bb, B, relres, st);
}

// Mixed precision: FP32-operator CG on the correction equation inside FP64
// iterative refinement, x += CG32(r), r = b - (K64 + lambda I) x.
static anova_status cg_mixed(anova_plan* plan, double lambda, const double* b, double* x, double tol, int maxit,
                             const CgBuffers& B, int* iters, double* relres, cudaStream_t st) {
    const int64_t N = plan->N;
    const double inner_tol = 1e-4;     // per refinement pass (tighter FP32 passes converge slowly near the floor)
    double* rhs = B.x2;            // current residual (right-hand side of the correction)
    double* dx = static_cast<double*>(nullptr);
    Scratch scratch(st);
    ANOVA_CUDA_TRY(scratch.alloc(&dx, std::max<int64_t>(N, 1) * sizeof(double)));
    ANOVA_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double), st));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(rhs, b, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_cg_init<<<B.nblk, kThreads, 0, st>>>(b, N, B.q, B.r, B.p, 0, B.part);
    k_reduce_to<<<1, kThreads, 0, st>>>(B.part, B.nblk, B.scal);
    double bb = 0.0;
    anova_status s = read_scalar(B.scal, &bb, st);
    int total = 0;
    double rel = 1.0;
    while (s == ANOVA_OK && bb > 0.0 && total < maxit) {
        int it = 0;
        double rb = 0.0;
        double tol_in = std::max(inner_tol, 0.5 * tol / std::max(rel, 1e-300));
        s = cg_run<float>(plan, lambda, rhs, dx, std::min(tol_in, 0.5), maxit - total, B, &it, &rb, st);
        if (s != ANOVA_OK) break;
        total += std::max(it, 1);
        k_axpy<<<grid_for(N, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(N, 1.0, dx, x);
        // FP64 residual of the original system
        s = apply_shifted<double>(plan, lambda, x, B.q, B, st);
        if (s != ANOVA_OK) break;
        k_residual<<<B.nblk, kThreads, 0, st>>>(b, B.q, N, rhs, B.part);
        k_reduce_to<<<1, kThreads, 0, st>>>(B.part, B.nblk, B.scal + 1);
        double rr = 0.0;
        s = read_scalar(B.scal + 1, &rr, st);
        if (s != ANOVA_OK) break;
        rel = std::sqrt(rr / bb);
        if (!std::isfinite(rel)) {
            set_error("refinement residual is not finite");
            s = ANOVA_ERANGE;
            break;
        }
        if (rel <= tol) break;
    }
    *iters = total;
    *relres = (bb > 0.0) ? rel : 0.0;
    if (s == ANOVA_OK && bb > 0.0 && rel > tol) s = ANOVA_ENOCONV;
    return s;
}

// ------------------------------------------------------------ debug spread
template <typename T>
static anova_status debug_spread_t(anova_plan* plan, int l, const void* alpha, void* grid, cudaStream_t st) {
    const WindowPlan& w = plan->win[l];
    size_t ge = 1;
    for (int t = 0; t < w.dA; t++) ge *= w.nos;
    ANOVA_CUDA_TRY(cudaMemsetAsync(grid, 0, ge * sizeof(T), st));
    return spread_window<T>(plan, w, w.X, alpha, sizeof(T) == 8, static_cast<T*>(grid), st);
}

// ---------------------------------------------------------------- predict
// Window l's part of the test-point summation (Sec. 4.3) at M test
// coordinates zw (device, this window's features): out = K_l(Z, X) alpha.
// Test points outside the plan's ball are summed in the joint frame of nodes
// and test points (window_reframe).  Uses the plan's grid of the window.
template <typename T>
anova_status predict_window(anova_plan* plan, int l, const double* alpha, const double* zw, int64_t M, T* out,
                            cudaStream_t st) {
    const WindowPlan& base = plan->win[l];
    double rmax = 0.0;
    ANOVA_TRY(max_radius(plan, zw, M, base.dA, base.centre, &rmax, st));
    WindowPlan joint;
    const bool reframe = base.scale * rmax > 0.25 - 0.5 * plan->epsB;
    anova_status s = ANOVA_OK;
    if (reframe) {
        s = window_reframe(plan, l, zw, M, joint, st);
        if (s != ANOVA_OK) {
            window_release_reframed(joint);
            return s;
        }
    }
    const WindowPlan& w = reframe ? joint : base;
    PointSet zs;
    WindowPlan wz = w;   // binning parameters of the window
    s = build_pointset(plan, wz, zw, M, w.dA, w.centre, w.scale, zs, st);
    size_t ge = 1;
    for (int t = 0; t < w.dA; t++) ge *= w.nos;
    T* grid = grid_of<T>(plan, w);
    if (s == ANOVA_OK && plan->N > 0) {
        cudaMemsetAsync(grid, 0, ge * sizeof(T), st);
        s = spread_window<T>(plan, w, w.X, alpha, 1, grid, st);
        if (s == ANOVA_OK) s = fft_convolve_window<T>(plan, w, grid, st);
        if (s == ANOVA_OK) s = gather_window<T>(plan, w, zs, grid, out, st);
    } else if (s == ANOVA_OK) {
        cudaMemsetAsync(out, 0, M * sizeof(T), st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == ANOVA_OK && e != cudaSuccess) {
        set_error(std::string("predict: ") + cudaGetErrorString(e));
        s = ANOVA_ECUDA;
    }
    free_pointset_async(zs, st);
    wz.X = PointSet();
    if (reframe) window_release_reframed(joint);
    return s;
}

template anova_status predict_window<double>(anova_plan*, int, const double*, const double*, int64_t, double*,
                                             cudaStream_t);
template anova_status predict_window<float>(anova_plan*, int, const double*, const double*, int64_t, float*,
                                            cudaStream_t);

template <typename T>
static anova_status predict_t(anova_plan* plan, const double* alpha, const double* Z, int64_t M, int64_t ldz,
                              double* out, cudaStream_t st) {
    const int P = plan->P;
    T* tmp = nullptr;
    double* zw = nullptr;
    Scratch scratch(st);
    ANOVA_CUDA_TRY(scratch.alloc(&tmp, std::max<int64_t>(M, 1) * P * sizeof(T)));
    ANOVA_CUDA_TRY(scratch.alloc(&zw, std::max<int64_t>(M, 1) * 3 * sizeof(double)));
    anova_status s = ANOVA_OK;
    for (int l = 0; l < P && s == ANOVA_OK; l++) {
        s = extract_window(plan, Z, M, ldz, plan->win[l], zw, st);
        if (s == ANOVA_OK) s = predict_window<T>(plan, l, alpha, zw, M, tmp + (int64_t)l * M, st);
    }
    if (s == ANOVA_OK && M > 0) {
        k_window_sum<T, double><<<grid_for(M, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            tmp, plan->eta_dev, P, M, out);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("predict: ") + cudaGetErrorString(e));
            s = ANOVA_ECUDA;
        }
    }
    return s;
}

}  // namespace anova

using namespace anova;

extern "C" {

anova_status anova_matvec(anova_plan* plan, int32_t dtype, const void* alpha, void* out, int32_t nrhs,
                          int64_t ld, void* stream) {
    if (!plan || !has_precision(plan, dtype) || nrhs < 1 || ld < plan->N ||
        (plan->N > 0 && (!alpha || !out))) {
        set_error("anova_matvec: bad plan, dtype, pointers, nrhs or ld");
        return ANOVA_EINVAL;
    }
    if (plan->N > 0 && alpha == out) {
        set_error("anova_matvec: out must not alias alpha");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (nrhs == 1 && plan->N > 0)
        return run_cached(plan, 0, dtype, alpha, out, 0.0, st, [&](cudaStream_t s) -> anova_status {
            if (dtype == ANOVA_FP64)
                return matvec_one<double>(plan, static_cast<const double*>(alpha), static_cast<double*>(out), s);
            return matvec_one<float>(plan, static_cast<const float*>(alpha), static_cast<float*>(out), s);
        });
    for (int r = 0; r < nrhs; r++) {
        if (dtype == ANOVA_FP64)
            ANOVA_TRY(matvec_one<double>(plan, static_cast<const double*>(alpha) + r * ld,
                                         static_cast<double*>(out) + r * ld, st));
        else
            ANOVA_TRY(matvec_one<float>(plan, static_cast<const float*>(alpha) + r * ld,
                                        static_cast<float*>(out) + r * ld, st));
    }
    return ANOVA_OK;
}

anova_status krr_cg_solve(anova_plan* plan, double lambda, const double* y, double* alpha, int32_t nrhs,
                          int64_t ld, double tol, int32_t maxit, int32_t* iters, double* relres,
                          void* stream) {
    if (!plan || !(lambda > 0.0) || !std::isfinite(lambda) || !(tol > 0.0) || maxit < 0 ||
        maxit > ANOVA_MAX_CG_ITERS || nrhs < 1 ||
        ld < plan->N || (plan->N > 0 && (!y || !alpha))) {
        set_error("krr_cg_solve: bad plan, lambda, tol, maxit, nrhs, ld or pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    anova_status worst = ANOVA_OK;
    if (plan->N == 0) {
        for (int r = 0; r < nrhs; r++) {
            if (iters) iters[r] = 0;
            if (relres) relres[r] = 0.0;
        }
        return ANOVA_OK;
    }
    CgBuffers B;
    ANOVA_TRY(cg_buffers(plan, maxit, B));
    const uint64_t waits0 = wait_timeouts_on(st);
    for (int c = 0; c < nrhs; c++) {
        const double* b = y + c * ld;
        double* x = alpha + c * ld;
        int it = 0;
        double rel = 0.0, bb = 0.0;
        anova_status s;
        if (plan->precision == ANOVA_MIXED) {
            s = cg_mixed(plan, lambda, b, x, tol, maxit, B, &it, &rel, st);
        } else if (plan->precision & ANOVA_FP64) {
            s = cg_run<double>(plan, lambda, b, x, tol, maxit, B, &it, &bb, st);
            if (s == ANOVA_OK) s = true_residual<double>(plan, lambda, b, x, bb, B, &rel, st);
            if (s == ANOVA_OK && it >= maxit && rel > tol) s = ANOVA_ENOCONV;
        } else {
            s = cg_run<float>(plan, lambda, b, x, tol, maxit, B, &it, &bb, st);
            if (s == ANOVA_OK) s = true_residual<float>(plan, lambda, b, x, bb, B, &rel, st);
            if (s == ANOVA_OK && it >= maxit && rel > tol) s = ANOVA_ENOCONV;
        }
        if (iters) iters[c] = it;
        if (relres) relres[c] = rel;
        if (s != ANOVA_OK && s != ANOVA_ENOCONV) return s;
        if (s == ANOVA_ENOCONV) worst = s;
    }
    if (wait_timeouts_on(st) != waits0) {
        set_error("krr_cg_solve: a bounded wait inside a kernel gave up during the solve");
        return ANOVA_ETIMEOUT;
    }
    return worst;
}

anova_status krr_predict(anova_plan* plan, const double* alpha, const double* Z, int64_t M, int64_t ldz,
                         double* out, void* stream) {
    if (!plan || M < 0 || M > INT32_MAX || ldz < plan->d || (M > 0 && (!Z || !out)) ||
        (plan->N > 0 && !alpha)) {
        set_error("krr_predict: bad plan, sizes or pointers");
        return ANOVA_EINVAL;
    }
    if (M == 0) return ANOVA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t w0 = wait_timeouts_on(st);
    const anova_status s = (plan->precision & ANOVA_FP64) ? predict_t<double>(plan, alpha, Z, M, ldz, out, st)
                                                          : predict_t<float>(plan, alpha, Z, M, ldz, out, st);
    return waits_moved(w0, st, "krr_predict", s);
}

anova_status anova_debug_spread(anova_plan* plan, int32_t l, int32_t dtype, const void* alpha, void* grid,
                                void* stream) {
    if (!plan || l < 0 || l >= plan->P || !has_precision(plan, dtype) || !grid ||
        (plan->N > 0 && !alpha)) {
        set_error("anova_debug_spread: bad arguments");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == ANOVA_FP64) return debug_spread_t<double>(plan, l, alpha, grid, st);
    return debug_spread_t<float>(plan, l, alpha, grid, st);
}

anova_status anova_set_profiling(anova_plan* plan, int32_t enable) {
    if (!plan) return ANOVA_EINVAL;
    plan->clock.enabled = enable != 0;
    return ANOVA_OK;
}

anova_status anova_plan_set_graphs(anova_plan* plan, int32_t enable) {
    if (!plan) return ANOVA_EINVAL;
    plan->use_graphs = enable != 0;
    if (!plan->use_graphs) {
        for (auto& g : plan->graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        plan->graphs.clear();
    }
    return ANOVA_OK;
}

anova_status anova_plan_set_tensor_cores(anova_plan* plan, int32_t enable) {
    if (!plan) return ANOVA_EINVAL;
    const bool on = enable != 0;
    plan->spread_tc = on;
    plan->gather_tc = on;
    plan->gather_umma = on;
    plan->gather_tc5 = on;
    plan->spread_tc5 = enable == 2;
    plan->spread_f16 = false;
    for (auto& g : plan->graphs)      // the captured launch sequences name the old kernels
        if (g.exec) cudaGraphExecDestroy(g.exec);
    plan->graphs.clear();
    return ANOVA_OK;
}

anova_status anova_plan_set_overlap(anova_plan* plan, int32_t mode) {
    if (!plan || mode < 0 || mode > 7 || ((mode & 3) == 0 && mode != 0)) {
        set_error("anova_plan_set_overlap: mode must be 0, 1..3 or 5..7");
        return ANOVA_EINVAL;
    }
    plan->overlap12 = mode;
    for (auto& g : plan->graphs)      // the captured launch sequences hold the old schedule
        if (g.exec) cudaGraphExecDestroy(g.exec);
    plan->graphs.clear();
    return ANOVA_OK;
}

int32_t anova_stage_times(anova_plan* plan, double* ms, int64_t* launches, int32_t cap) {
    if (!plan) return 0;
    StageClock& c = plan->clock;
    for (size_t i = 0; i + 1 < c.ev.size(); i += 2) {
        cudaEventSynchronize(c.ev[i + 1]);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c.ev[i], c.ev[i + 1]) == cudaSuccess) c.ms[c.stage_of_pair[i / 2]] += t;
        cudaEventDestroy(c.ev[i]);
        cudaEventDestroy(c.ev[i + 1]);
    }
    c.ev.clear();
    c.stage_of_pair.clear();
    for (int& o : c.open) o = -1;
    int k = std::min<int>(cap, StageClock::kStages);
    for (int i = 0; i < k; i++) {
        if (ms) ms[i] = c.ms[i];
        if (launches) launches[i] = c.launches[i];
        c.ms[i] = 0.0;
        c.launches[i] = 0;
    }
    return k;
}

}  // extern "C"
