// noalloc.cu -- krr_predict_noalloc: prediction at test points without any
// device allocation.
//
// krr_predict needs per-call scratch for the test points (their window
// coordinates, the binned and sorted copy, the sort's histograms and the
// per-window results) and gets it from cudaMalloc.  Some callers cannot
// allocate inside the call: a server that keeps a fixed device-memory
// footprint under an admission budget, or a host process whose allocator is
// owned by another framework.  This variant takes that scratch from one
// file-scope device array instead.  The plan's own buffers (grid, FFT work
// arrays, the binned training nodes), created once by anova_fastsum_plan, are
// used as before.  The call synchronises its stream: the ball check reads each
// window's largest test-point radius back to the host.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace anova {

// Capacity: at most kNoallocMaxPoints test points per call.
constexpr int64_t kNoallocMaxPoints = 65536;
constexpr size_t kNoallocScratchBytes = 8u << 20;   // 8 MiB, held by every GPU that loads the library

static __device__ __align__(256) unsigned char g_predict_scratch[kNoallocScratchBytes];

// Device address of g_predict_scratch, looked up once per device with that
// device current.  In host code the symbol itself is only a host-side stand-in.
static void* scratch_address(anova_status* status) {
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_error(std::string("krr_predict_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        *status = ANOVA_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_predict_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("krr_predict_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            *status = ANOVA_ECUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    *status = ANOVA_OK;
    return addr[dev];
}

// out = (first ? 0 : out) + eta * tmp
template <typename T>
__global__ void k_accumulate(const T* __restrict__ tmp, double eta, int64_t M, int first, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (first ? 0.0 : out[i]) + eta * (double)tmp[i];
}

struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <typename T>
    T* take(int64_t n) {
        used = (used + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + used);
        used += (size_t)n * sizeof(T);
        return p;
    }
};

template <typename T>
static anova_status predict_noalloc_t(anova_plan* plan, const double* alpha, const double* Z, int64_t M,
                                      int64_t ldz, double* out, unsigned char* scratch, cudaStream_t st) {
    NoallocBinBuffers buf = noalloc_bin_layout(M);
    Carver cv{scratch};
    double* zw = cv.take<double>(3 * M);
    T* tmp = cv.take<T>(M);
    buf.perm = cv.take<int32_t>(M);
    buf.cell = cv.take<int32_t>(3 * M);
    buf.frac64 = cv.take<double>(3 * M);
    buf.frac32 = cv.take<float>(3 * M);
    buf.bin_start = cv.take<int32_t>(kMaxBins + 1);
    buf.nch = cv.take<int32_t>(kMaxBins + 1);
    buf.hist = cv.take<int32_t>(buf.hist_elems);
    buf.tot = cv.take<int32_t>(2);
    buf.sub = cv.take<int4>(buf.sub_capacity);
    double* red = cv.take<double>(buf.red_elems);
    if (cv.used > kNoallocScratchBytes) {
        set_error("krr_predict_noalloc: scratch layout exceeds the static array");
        return ANOVA_EINVAL;
    }
    const double RB = 0.25 - 0.5 * plan->epsB;
    for (int l = 0; l < plan->P; l++) {
        WindowPlan& w = plan->win[l];
        ANOVA_TRY(extract_window(plan, Z, M, ldz, w, zw, st));
        double rmax = 0.0;
        ANOVA_TRY(max_radius_into(plan, zw, M, w.dA, w.centre, red, &rmax, st));
        if (w.scale * rmax > RB) {
            set_error("krr_predict_noalloc: a test point lies outside the plan's ball in window " +
                      std::to_string(l) + " (krr_predict handles this case by re-framing)");
            return ANOVA_ERANGE;
        }
        PointSet zs;
        ANOVA_TRY(build_pointset_into(plan, w, zw, M, w.centre, w.scale, buf, zs, st));
        size_t ge = 1;
        for (int t = 0; t < w.dA; t++) ge *= w.nos;
        T* grid = grid_of<T>(plan, w);
        if (plan->N > 0) {
            ANOVA_CUDA_TRY(cudaMemsetAsync(grid, 0, ge * sizeof(T), st));
            ANOVA_TRY(spread_window<T>(plan, w, w.X, alpha, 1, grid, st));
            ANOVA_TRY(fft_convolve_window<T>(plan, w, grid, st));
            ANOVA_TRY(gather_window<T>(plan, w, zs, grid, tmp, st));
        } else {
            ANOVA_CUDA_TRY(cudaMemsetAsync(tmp, 0, M * sizeof(T), st));
        }
        k_accumulate<T><<<grid_for(M, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(tmp, w.eta, M, l == 0, out);
        ANOVA_CHECK_LAUNCH();
    }
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

}  // namespace anova

using namespace anova;

extern "C" anova_status krr_predict_noalloc(anova_plan* plan, const double* alpha, const double* Z, int64_t M,
                                            int64_t ldz, double* out, void* stream) {
    if (!plan || M < 0 || ldz < plan->d || (M > 0 && (!Z || !out)) || (plan->N > 0 && !alpha)) {
        set_error("krr_predict_noalloc: bad plan, sizes or pointers");
        return ANOVA_EINVAL;
    }
    if (M > kNoallocMaxPoints) {
        set_error("krr_predict_noalloc: at most 65536 test points per call");
        return ANOVA_EINVAL;
    }
    if (M == 0) return ANOVA_OK;
    anova_status s = ANOVA_OK;
    unsigned char* scratch = static_cast<unsigned char*>(scratch_address(&s));
    if (s != ANOVA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->precision & ANOVA_FP64) return predict_noalloc_t<double>(plan, alpha, Z, M, ldz, out, scratch, st);
    return predict_noalloc_t<float>(plan, alpha, Z, M, ldz, out, scratch, st);
}
