// common.cuh -- internal types and device helpers of libanova_gb300.
//
// Notation (arXiv 2111.10140, Sec. 4): window l has dA in {1,2,3} features,
// bandwidth n, oversampled grid nos = sigma*n per axis, Kaiser-Bessel cutoff m.
// Grid and frequency arrays use the centred index of I_M (value v stored at
// v + M/2), last axis fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/anova_gb300.h"

namespace anova {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
#define ANOVA_CUDA_TRY(expr)                                                    \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) {                                                \
            ::anova::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
            return ANOVA_ECUDA;                                                 \
        }                                                                       \
    } while (0)
#define ANOVA_TRY(expr)                       \
    do {                                      \
        anova_status _s = (expr);             \
        if (_s != ANOVA_OK) return _s;        \
    } while (0)
#define ANOVA_CHECK_LAUNCH() ANOVA_CUDA_TRY(cudaGetLastError())

// ------------------------------------------------------ device allocation
// Every device allocation of the library goes through these two calls.  A
// host-side hook (anova_debug_fail_alloc) can make the k-th one fail, to test
// the error paths without a device fault.
cudaError_t dev_malloc(void** ptr, size_t bytes);
cudaError_t dev_malloc_async(void** ptr, size_t bytes, cudaStream_t st);

// The device scratch of one call: freed (stream-ordered when `async`) when the
// guard leaves scope, on every exit path, unless handed to an owner first.
struct Scratch {
    cudaStream_t st = nullptr;
    bool async = true;
    std::vector<void*> ptrs;
    Scratch(cudaStream_t s, bool a = true) : st(s), async(a) {}
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    template <typename T>
    cudaError_t alloc(T** p, size_t bytes) {
        void* v = nullptr;
        const cudaError_t e = async ? dev_malloc_async(&v, bytes, st) : dev_malloc(&v, bytes);
        *p = static_cast<T*>(v);
        if (e == cudaSuccess && v) ptrs.push_back(v);
        return e;
    }
    void keep(const void* p) {   // ownership passes to the caller's structure
        for (auto& q : ptrs)
            if (q == p) q = nullptr;
    }
    ~Scratch() {
        for (void* p : ptrs)
            if (p) {
                if (async) cudaFreeAsync(p, st);
                else cudaFree(p);
            }
    }
};

// ------------------------------------------------------------- constants
constexpr int kMaxDim = 3;
constexpr int kMaxWindows = 256;
constexpr int kMaxM = 12;
constexpr int kSubChunk = 256;         // points per spread/gather sub-problem
constexpr int kThreads = 256;
constexpr int kMaxBins = 32768;        // bins per window (shared histogram of the sort)
constexpr int kPsiDeg = 8;             // degree of the per-interval window polynomials (FP32 path)
constexpr int kPsiStride = kPsiDeg + 1;

// Points of one window, binned and sorted (one for the training nodes X,
// one per predict call for the test nodes Z).
struct PointSet {
    int64_t N = 0;
    int32_t* perm = nullptr;       // sorted position -> original index
    int32_t* cell = nullptr;       // dA x N cell index per axis in [0, nos)
    double* frac64 = nullptr;      // dA x N, nos*x - floor(nos*x) in FP64
    float* frac32 = nullptr;       // dA x N, same rounded to FP32
    int32_t* bin_start = nullptr;  // nbins + 1 offsets of each bin in sorted order
    int4* sub = nullptr;           // sub-problems: (bin, first, count, 0)
    int32_t nsub = 0;
};

struct WindowPlan {
    int dA = 0;
    int feat[kMaxDim] = {-1, -1, -1};
    int n = 0, nos = 0;
    int T = 0;        // bin side in grid cells
    int nb = 0;       // bins per axis, ceil(nos / T)
    int R = 0;        // region side = T + 2m
    int nbins = 0;    // nb^dA
    bool dense = false;  // 3-D window on the dense tensor-product kernels (dense3.cu)
    double eta = 0.0;
    double centre[kMaxDim] = {0, 0, 0};
    double scale = 1.0, ell_l = 0.0;
    double* D64 = nullptr;     // n^dA multiplier (FP64)
    float* D32 = nullptr;      // same in FP32
    double2* tw64 = nullptr;   // exp(-2 pi i r / nos), r = 0..nos-1
    float2* tw32 = nullptr;
    double* xw = nullptr;      // N x dA window coordinates (user units, original order)
    size_t grid_off = 0;       // element offset of this window's grid in plan->grid
    size_t work_off = 0;       // element offset of this window's FFT work arrays
    float* wtab = nullptr;     // dense 3-D windows, FP32 plans: N x 3 x 16 zero-padded window weights (sorted order)
    double* wtap64 = nullptr;  // FP64 plans: N x dA x (2m+1) window taps psi(m - k + f) of the nodes (sorted order)
    int box_lo[kMaxDim] = {0, 0, 0};   // grid cells touched by the training nodes: start (may be < 0)
    int box_ext[kMaxDim] = {0, 0, 0};  // and extent per axis (<= nos)
    bool fft12 = false;        // 1-D / 2-D window on the batched box FFT (fft12.cu)
    PointSet X;
};

// Per-window arguments of the batched box-restricted 1-D / 2-D FFT (fft12.cu).
struct Fft12Win {
    void* grid;                // real grid, nos^dA
    const void* tw;            // e^{-2 pi i r/nos}
    const void* D;             // n^dA multiplier
    int dA, n, nos;
    int lo[2], B[2];           // box start and extent per axis
    const int* live = nullptr;   // batches: the instance's system still iterates (null: always)
};
constexpr size_t kFft12MaxSmem = 227 * 1024;

// Per-window arguments of the batched box-restricted 3-D FFT (fft3.cu).
struct Fft3Win {
    void* grid;                // real grid, nos^3
    void* buf1;                // complex work arrays
    void* buf2;
    const void* tw;            // e^{-2 pi i r/nos}
    const void* D;             // n^3 multiplier
    int lo[3], B[3];           // box start and extent per axis
    int n, nos;
    const int* live = nullptr;   // batches: the instance's system still iterates (null: always)
};

// Per-window arguments of the batched dense 3-D kernels (one launch, all windows).
struct DenseWin {
    const int32_t* perm;
    const int32_t* cell;
    const void* frac;          // FP32 or FP64, as the launch
    const float* wtab;         // FP32 weight table (N x 48) or null
    const double* wtap = nullptr;   // FP64 tap table of the plan's nodes (N x 3 x (2m+1)) or null
    float* asort;              // FP32 coefficients in this window's sorted order (filled per matvec)
    void* grid;                // this window's grid
    void* out;                 // gather output (this window's slice of plan->tmp)
    int64_t N;
    int nos, Tb, nb, pad;
    const int* live = nullptr;   // batches: the instance's system still iterates (null: always)
};

struct StageClock {
    bool enabled = false;
    // 0 spread, 1 FFT / multiply / inverse FFT, 2 gather, 3 window sum and CG vectors;
    // 4 and 5 time the 3-D spread and 3-D gather launches alone (inside stages 0 and 2)
    static constexpr int kStages = 6;
    std::vector<cudaEvent_t> ev;       // pairs (start, stop)
    std::vector<int> stage_of_pair;
    double ms[kStages] = {0, 0, 0, 0, 0, 0};
    int64_t launches[kStages] = {0, 0, 0, 0, 0, 0};
    int open[kStages] = {-1, -1, -1, -1, -1, -1};   // index in ev of the stage's open start event
};

}  // namespace anova

struct anova_plan {
    int64_t N = 0;
    int d = 0, P = 0, m = 0, p = 0, precision = 0;
    double sigma = 2.0, epsB = 1.0 / 16, ell = 0.0, b = 0.0;
    double psi_norm = 1.0;              // m / sinh(b m): psi(t) = psi_norm * sinh(b s)/s
    float* psi_poly = nullptr;          // 2m x kPsiStride: psi(q - m + f) ~ sum_k c_k (f - 1/2)^k; then psi(m)
    double* psi_poly64 = nullptr;       // the same coefficients in FP64 (the FP32 weight tables)
    std::vector<anova::WindowPlan> win;
    // work buffers: every window has its own grid and FFT work arrays (offsets in WindowPlan)
    size_t grid_elems = 0, work_elems = 0;  // totals over the windows
    void* grid = nullptr;               // real spread grids / inverse FFT outputs
    void* work1 = nullptr;              // complex work arrays
    void* work2 = nullptr;
    // batched dense 3-D windows: merged sub-problem list (bin, first, count, window)
    int4* dense_sub = nullptr;
    int dense_nsub = 0;
    std::vector<int> dense_windows;     // indices of the dense windows, in launch order
    std::vector<std::array<int, 3>> dense_groups;  // (region size R, first sub, count) per launch
    anova::DenseWin* dense_desc = nullptr;  // device, 2 x dense_windows.size(): FP64 then FP32
    float* dense_asort = nullptr;       // dense_windows.size() x N sorted FP32 coefficients
    bool spread_tc = true;              // FP32 dense spread on tensor cores (3xTF32) instead of FFMA2
    bool spread_pipe = true;            // ... with the next chunk's rows copied (cp.async) during the current MMAs
    bool spread_f16 = false;            // ... as FP16-split m16n8k16 MMAs (coefficients scaled by max |alpha|)
    unsigned* f16_scale = nullptr;      // device word: bits of max |alpha| for that form
    int overlap12 = 1;                  // FP32 product: the 1-D / 2-D windows on a second stream beside the 3-D
                                        // ones (anova_plan_set_overlap: 0 off, 1 forked before the 3-D spread,
                                        // 2 after the 3-D spread is queued, 3 after it has run; +4 high priority)
    cudaStream_t side = nullptr;        // that stream (created with the plan, lowest priority)
    cudaStream_t side_hi = nullptr;     // the same at the highest priority
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool gather_tc = true;              // FP32 dense gather on tensor cores (3xTF32) instead of FFMA2
    bool gather_umma = true;            // ... on tcgen05 (tensor memory accumulators) instead of mma.sync
    bool gather_tc5 = true;             // FP32 dense 3-D gather: persistent tcgen05 kernel, weights on the fly
    bool pw12 = true;                   // FP32 dense 1-D / 2-D kernels: persistent, weights on the fly
    bool spread_tc5 = false;            // FP32 dense 3-D spread: persistent tcgen05 kernel (A in tensor memory); measured slower
    std::vector<float> psi_host;        // host copy of psi_poly (kernel parameters of the persistent kernels)
    int bin_side[3] = {0, 0, 0};        // bin side of the dense 1-D / 2-D / 3-D windows (0: the default rule)
    std::vector<int> fft3_windows;      // 3-D windows on the batched box FFT
    anova::Fft3Win* fft3_desc = nullptr;    // device, 2 x fft3_windows.size(): FP64 then FP32
    bool fft3_slab = false;             // every batched 3-D window fits the slab kernels
    std::vector<int> fft12_windows;     // 1-D / 2-D windows on the batched box FFT
    anova::Fft12Win* fft12_desc = nullptr;  // device, 2 x fft12_windows.size(): FP64 then FP32
    size_t fft12_smem64 = 0, fft12_smem32 = 0;   // dynamic shared memory of the launch
    int fft12_uniform_n = 0;            // n of every such window when all share it with n_os = 2 n, else 0
    void* tmp = nullptr;                // P x N per-window results (8 bytes each)
    double* eta_dev = nullptr;          // P window weights on the device
    // CG state
    double* cg_vec = nullptr;           // r, p, q, a (FP64), each N
    double* cg_scal = nullptr;          // scalars and per-iteration history
    double* cg_part = nullptr;          // block partial sums
    int cg_hist = 0;
    anova::StageClock clock;
    int sm_count = 0;
    // replayable launch sequences of anova_matvec, keyed by (dtype, alpha, out)
    struct GraphEntry {
        int kind;            // 0: anova_matvec, 1: CG operator application
        int dtype;
        const void* alpha;
        void* out;
        double lambda;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t capture_stream = nullptr;
    bool use_graphs = true;
};

namespace anova {

// ------------------------------------------------------------ device math
// Kaiser-Bessel window normalised to psi(0) = 1 (grid units t):
//   psi(t) = (m / sinh(b m)) * sinh(b s) / s,  s = sqrt(m^2 - t^2), |t| <= m,
// with the limit (m / sinh(b m)) * b at |t| = m and 0 beyond.
template <typename T>
__device__ __forceinline__ T kb_psi(T t, T m, T b, T norm) {
    T s2 = m * m - t * t;
    if (s2 < T(0)) return T(0);
    T s = sqrt(s2);
    T r = (s > T(0)) ? sinh(b * s) / s : b;
    return norm * r;
}

// FP32 window weight from the per-interval polynomials: t = j + f with integer
// j and f in [0, 1); zero outside [-m, m], psi(m) (kept after the 2m rows of
// coefficients) at the closed end t = m.
__device__ __forceinline__ float psi_poly_eval(const float* __restrict__ P, int j, float f, int m) {
    const int q = j + m;
    if (q == 2 * m) return f == 0.f ? P[2 * m * kPsiStride] : 0.f;
    if (q < 0 || q > 2 * m) return 0.f;
    const float* c = P + q * kPsiStride;
    const float u = f - 0.5f;
    float acc = c[kPsiDeg];
#pragma unroll
    for (int k = kPsiDeg - 1; k >= 0; k--) acc = fmaf(acc, u, c[k]);
    return acc;
}

// ------------------------------------------------------------- host API
anova_status build_pointset(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                            int64_t ldc, const double* centre, double scale, PointSet& ps,
                            cudaStream_t st);
void free_pointset(PointSet& ps);
void free_pointset_async(PointSet& ps, cudaStream_t st);
anova_status window_reframe(anova_plan* plan, int l, const double* zw, int64_t M, WindowPlan& dst,
                            cudaStream_t st);
template <typename T>
anova_status predict_window(anova_plan* plan, int l, const double* alpha, const double* zw, int64_t M, T* out,
                            cudaStream_t st);
anova_status window_widened(anova_plan* plan, int l, double rho, WindowPlan& dst, cudaStream_t st);
void window_release_reframed(WindowPlan& w);
anova_status max_radius(anova_plan* plan, const double* zw, int64_t M, int dA, const double* centre,
                        double* rmax_host, cudaStream_t st);
anova_status extract_window(anova_plan* plan, const double* Z, int64_t M, int64_t ldz,
                            const WindowPlan& w, double* zw, cudaStream_t st);

// caller-provided buffers for binning M nodes without allocating
struct NoallocBinBuffers {
    int nchunk = 0;              // capacity in node chunks of the sort
    int64_t hist_elems = 0;      // capacity of hist
    int sub_capacity = 0;        // capacity of sub
    int64_t red_elems = 0;       // capacity of the radius reduction buffer
    int32_t* perm = nullptr;     // M
    int32_t* cell = nullptr;     // 3 M
    double* frac64 = nullptr;    // 3 M
    float* frac32 = nullptr;     // 3 M
    int32_t* bin_start = nullptr;// kMaxBins + 1
    int32_t* nch = nullptr;      // kMaxBins + 1
    int32_t* hist = nullptr;     // hist_elems
    int32_t* tot = nullptr;      // 2
    int4* sub = nullptr;         // sub_capacity
};
NoallocBinBuffers noalloc_bin_layout(int64_t M);
anova_status max_radius_into(anova_plan* plan, const double* zw, int64_t M, int dA, const double* centre,
                             double* red, double* rmax_host, cudaStream_t st);
anova_status build_pointset_into(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                                 const double* centre, double scale, const NoallocBinBuffers& buf,
                                 PointSet& ps, cudaStream_t st);

// window-level stages (matvec.cu / spread_gather.cu / fft.cu)
template <typename T>
anova_status spread_window(anova_plan* plan, const WindowPlan& w, const PointSet& ps,
                           const void* alpha, int alpha_is_double, T* grid, cudaStream_t st);
template <typename T>
anova_status gather_window(anova_plan* plan, const WindowPlan& w, const PointSet& ps,
                           const T* h, T* out, cudaStream_t st);
template <typename T>
anova_status spread3_dense(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const void* alpha,
                           int alpha_double, T* grid, cudaStream_t st);
template <typename T>
anova_status gather3_dense(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const T* h, T* out,
                           cudaStream_t st);
template <typename T>
anova_status fft_convolve_window(anova_plan* plan, const WindowPlan& w, T* grid, cudaStream_t st);
template <typename T>
anova_status fft3_box_all(anova_plan* plan, cudaStream_t st);
bool fft3_box_supported(const WindowPlan& w);
template <typename T>
anova_status fft12_box_all(anova_plan* plan, cudaStream_t st);
bool fft12_box_supported(const WindowPlan& w);
template <typename T>
anova_status fft12_box_run(const Fft12Win* desc, int nw, size_t smem, cudaStream_t st, int uniform_n);
anova_status gather3_umma(int R, const int4* sub, int nsub, const DenseWin* descs, int m, const float* poly,
                          cudaStream_t st);
// plain FP64 CG from x = 0 on a plan holding FP64 data (matvec.cu)
anova_status cg_fp64_solve(anova_plan* plan, double lambda, const double* b, double* x, double tol, int maxit,
                           int* iters, double* relres, cudaStream_t st);
// persistent tcgen05 3-D kernels (tc3.cu): (R, m) pairs built, and the launches
bool tc5_supported(int R, int m);
// the persistent gather pays off once every SM has enough tiles to fill its pipeline
inline bool tc5_gather_pays(int nsub, int sms) { return 2 * (int64_t)nsub >= 48 * (int64_t)sms; }
anova_status gather3_tc5(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const float* psi_host,
                         int sms, cudaStream_t st);
anova_status spread3_tc5(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const float* psi_host,
                         int sms, const void* alpha, int alpha_double, cudaStream_t st);
anova_status spread3_f16(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const void* alpha,
                         int alpha_double, int64_t N, unsigned* scale, int sms, cudaStream_t st);
// persistent FP32 1-D / 2-D kernels with on-the-fly weights (dense12.cu)
anova_status dense12_pw(int dA, bool spread, int R, int m, const int4* sub, int nsub, const DenseWin* descs,
                        const float* psi_host, int sms, const void* alpha, int alpha_double, cudaStream_t st);
uint64_t wait_timeouts_on(cudaStream_t st);
// s, or ETIMEOUT when the wait counter moved since `before` (the call's result
// is then invalid); synchronises st
anova_status waits_moved(uint64_t before, cudaStream_t st, const char* who, anova_status s);
anova_status dense_f32_spread_groups(int m, const int4* sub_base, const DenseWin* descs,
                                     const std::vector<std::array<int, 3>>& groups, cudaStream_t st,
                                     const float* psi_host = nullptr, int sms = 0, bool tc5_3d = false);
anova_status dense_f32_gather_groups(int m, const float* poly, const int4* sub_base, const DenseWin* descs,
                                     const std::vector<std::array<int, 3>>& groups, cudaStream_t st,
                                     const float* psi_host = nullptr, int sms = 0);
// Shapes of a batched 3-D box FFT launch (maxima over its windows).
struct Fft3Shape {
    int nw = 0, nmax = 0, nosmax = 0, bx = 0, by = 0, bz = 0;
    int uniform_n = 0;         // n of every window when all share it with n_os = 2 n, else 0
    int64_t t1 = 0, t2 = 0, t3 = 0;
    bool slab = true;
    void add(const WindowPlan& w);
};
template <typename T>
anova_status fft3_box_run(const Fft3Win* wins, const Fft3Shape& sh, int sm_count, cudaStream_t st);
size_t fft12_window_smem(const WindowPlan& w, size_t real_bytes);
bool fft3_slab_supported(const WindowPlan& w);
// which dense groups a dense3_*_all call launches (and whether the spread sorts the coefficients first)
constexpr int kDense12 = 1, kDense3 = 2, kDenseSort = 4, kDenseAll = 7;
template <typename T>
anova_status dense3_spread_all(anova_plan* plan, const void* alpha, int alpha_double, cudaStream_t st,
                              int* launches = nullptr, int dims = kDenseAll);
template <typename T>
anova_status dense3_gather_all(anova_plan* plan, cudaStream_t st, int dims = kDenseAll);

template <typename T>
inline T* grid_of(anova_plan* plan, const WindowPlan& w) {
    return static_cast<T*>(plan->grid) + w.grid_off;
}

// stage clock helpers
void clock_begin(anova_plan* plan, int stage, cudaStream_t st);
void clock_end(anova_plan* plan, int stage, int launches, cudaStream_t st);

inline int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace anova
