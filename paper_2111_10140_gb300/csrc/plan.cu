// plan.cu -- plan construction for the ANOVA fast summation (arXiv 2111.10140).
//
//   A0  node scaling: per window, centre = bounding-box midpoint and
//       scale = (1/4 - eps_B/2) / max ||x - centre||, so scaled nodes lie in the
//       ball that keeps all pairwise distances below 1/2 - eps_B (Sec. 4.2,
//       "scaled nodes h^{-1} x", torus T = [-1/2, 1/2), Sec. 4.1).
//   A1  binning: a stable counting sort of each window's nodes by spatial bin
//       of T^dA grid cells, plus the list of sub-problems (bin, first, count)
//       that the spread and gather kernels walk.
//   A2  multiplier: b_k = n^{-dA} sum_{j in I_n} K_R(||j||/n) e^{-2 pi i k.j/n}
//       (Sec. 4.2, Fourier coefficients from equispaced samples of the
//       periodised kernel), divided by the squared Kaiser-Bessel transform
//       per axis (the window deconvolution of the adjoint NFFT and the NFFT).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"

namespace anova {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// ===================================================================== A0
// block-wide reductions over doubles (blockDim.x == kThreads)
__device__ double block_reduce_min(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : INFINITY;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}
__device__ double block_reduce_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : -INFINITY;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

// gather the window's columns: xw[i*dA + t] = X[i*ld + feat[t]]
__global__ void k_extract(const double* __restrict__ X, int64_t N, int64_t ld, int dA, int f0,
                          int f1, int f2, double* __restrict__ xw) {
    int feat[3] = {f0, f1, f2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < dA; t++) xw[i * dA + t] = X[i * ld + feat[t]];
}

// per-block min/max per axis over two point sets (a: Na x dA, b: Nb x dA)
__global__ void k_minmax(const double* __restrict__ a, int64_t Na, const double* __restrict__ b,
                         int64_t Nb, int dA, double* __restrict__ part) {
    __shared__ double sh[32];
    for (int t = 0; t < dA; t++) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Na + Nb;
             i += (int64_t)gridDim.x * blockDim.x) {
            double v = (i < Na) ? a[i * dA + t] : b[(i - Na) * dA + t];
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
        lo = block_reduce_min(lo, sh);
        hi = block_reduce_max(hi, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x * 6 + 2 * t] = lo;
            part[blockIdx.x * 6 + 2 * t + 1] = hi;
        }
    }
}

// frame[0..2] = centre, frame[3] = scale (filled by k_maxnorm_final)
__global__ void k_minmax_final(const double* __restrict__ part, int nblk, int dA,
                               double* __restrict__ frame) {
    __shared__ double sh[32];
    for (int t = 0; t < 3; t++) {
        double lo = INFINITY, hi = -INFINITY;
        if (t < dA)
            for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
                lo = fmin(lo, part[i * 6 + 2 * t]);
                hi = fmax(hi, part[i * 6 + 2 * t + 1]);
            }
        lo = block_reduce_min(lo, sh);
        hi = block_reduce_max(hi, sh);
        if (threadIdx.x == 0) frame[t] = (t < dA) ? 0.5 * (lo + hi) : 0.0;
    }
}

__global__ void k_maxnorm(const double* __restrict__ a, int64_t Na, const double* __restrict__ b,
                          int64_t Nb, int dA, const double* __restrict__ frame,
                          double* __restrict__ part) {
    __shared__ double sh[32];
    double c0 = frame[0], c1 = frame[1], c2 = frame[2];
    double best = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Na + Nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double* x = (i < Na) ? a + i * dA : b + (i - Na) * dA;
        double r2 = 0.0, df;
        df = x[0] - c0;
        r2 = df * df;
        if (dA > 1) { df = x[1] - c1; r2 += df * df; }
        if (dA > 2) { df = x[2] - c2; r2 += df * df; }
        best = fmax(best, r2);
    }
    best = block_reduce_max(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void k_maxnorm_final(const double* __restrict__ part, int nblk, double RB,
                                double* __restrict__ frame) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) best = fmax(best, part[i]);
    best = block_reduce_max(best, sh);
    if (threadIdx.x == 0) {
        double r = sqrt(best);
        frame[3] = (r > 0.0) ? RB / r : 1.0;
        frame[4] = r;
    }
}

// Frame of one window over one or two coordinate sets (device, n x dA each).
// frame_host receives centre[3], scale, max radius.
static anova_status compute_frame(anova_plan* plan, const double* a, int64_t Na, const double* b,
                                  int64_t Nb, int dA, double* scratch, double* frame_host,
                                  cudaStream_t st) {
    const int nblk = grid_for(Na + Nb, kThreads, 2 * std::max(plan->sm_count, 1));
    double* part = scratch;              // nblk * 6
    double* frame = scratch + 6 * nblk;  // 5
    k_minmax<<<nblk, kThreads, 0, st>>>(a, Na, b, Nb, dA, part);
    k_minmax_final<<<1, kThreads, 0, st>>>(part, nblk, dA, frame);
    k_maxnorm<<<nblk, kThreads, 0, st>>>(a, Na, b, Nb, dA, frame, part);
    k_maxnorm_final<<<1, kThreads, 0, st>>>(part, nblk, 0.25 - 0.5 * plan->epsB, frame);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemcpyAsync(frame_host, frame, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// ===================================================================== A1
// Bins: a node in grid cell c (per axis) belongs to bin c / T.  Blocks of one
// warp walk fixed chunks of nodes in order, which makes the sort stable.
constexpr int kBinChunk = 8192;

__device__ __forceinline__ void node_cell(const double* x, int dA, const double* c, double s,
                                          int nos, int* cell, double* frac) {
    for (int t = 0; t < dA; t++) {
        double xt = s * (x[t] - c[t]);           // torus coordinate
        double y = (double)nos * xt;             // grid units
        double fl = floor(y);
        frac[t] = y - fl;
        int ci = (int)fl + nos / 2;
        ci %= nos;
        if (ci < 0) ci += nos;
        cell[t] = ci;
    }
}

__device__ __forceinline__ int bin_of(const int* cell, int dA, int T, int nb) {
    int bin = 0;
    for (int t = 0; t < dA; t++) bin = bin * nb + cell[t] / T;
    return bin;
}

struct FrameArgs {
    double c[3];
    double s;
};

// per-chunk histograms, bin-major: hist[bin * nchunk + chunk]
__global__ void k_bin_hist(const double* __restrict__ xw, int64_t N, int dA, FrameArgs fr, int nos,
                           int T, int nb, int nbins, int nchunk, int32_t* __restrict__ hist) {
    extern __shared__ int32_t sh_hist[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    int64_t lo = (int64_t)blockIdx.x * kBinChunk, hi = min(N, lo + kBinChunk);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        int cell[3];
        double frac[3];
        node_cell(xw + i * dA, dA, fr.c, fr.s, nos, cell, frac);
        atomicAdd(&sh_hist[bin_of(cell, dA, T, nb)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        hist[(int64_t)i * nchunk + blockIdx.x] = sh_hist[i];
}

// single-block exclusive scan of L int32 values in place; total -> *total
__global__ void k_scan_exclusive(int32_t* __restrict__ v, int64_t L, int32_t* __restrict__ total) {
    __shared__ int32_t sh[1024];
    const int nt = blockDim.x;
    int64_t per = (L + nt - 1) / nt;
    int64_t lo = threadIdx.x * per, hi = min(L, lo + per);
    int32_t sum = 0;
    for (int64_t i = lo; i < hi; i++) sum += v[i];
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int32_t add = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    int32_t run = sh[threadIdx.x] - sum;
    for (int64_t i = lo; i < hi; i++) {
        int32_t x = v[i];
        v[i] = run;
        run += x;
    }
    if (threadIdx.x == nt - 1 && total) *total = sh[nt - 1];
}

// Multi-block exclusive scan for long histograms (bins x chunks of a large
// point set): tile sums, a single-block scan of the tile sums, then every
// tile scanned in shared memory from its offset.  Same result as
// k_scan_exclusive (integer sums), in three launches that fill the GPU.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const int32_t* __restrict__ v, int64_t L,
                                                                  int32_t* __restrict__ tsum) {
    __shared__ int32_t wsum[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t s = 0;
    for (int k = 0; k < kScanPer; k++) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < L) s += v[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = wsum[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) tsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int32_t* __restrict__ v, int64_t L,
                                                              const int32_t* __restrict__ toff) {
    __shared__ int32_t tile[kScanTile];
    __shared__ int32_t wsum[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int k = 0; k < kScanPer; k++) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < L ? v[i] : 0;
    }
    __syncthreads();
    // thread t owns the kScanPer consecutive values from t * kScanPer
    int32_t own[kScanPer];
    int32_t s = 0;
    for (int k = 0; k < kScanPer; k++) {
        own[k] = tile[threadIdx.x * kScanPer + k];
        s += own[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = s;                                   // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t x = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        wsum[lane] = x;                                // inclusive over warps
    }
    __syncthreads();
    int32_t run = toff[blockIdx.x] + (warp > 0 ? wsum[warp - 1] : 0) + inc - s;
    for (int k = 0; k < kScanPer; k++) {
        tile[threadIdx.x * kScanPer + k] = run;
        run += own[k];
    }
    __syncthreads();
    for (int k = 0; k < kScanPer; k++) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < L) v[i] = tile[k * kScanThreads + threadIdx.x];
    }
}

// exclusive scan of v[0, L) in place, total -> *total (device)
static anova_status scan_exclusive(int32_t* v, int64_t L, int32_t* total, Scratch& scratch, cudaStream_t st) {
    if (L <= 4 * kScanTile) {
        k_scan_exclusive<<<1, 1024, 0, st>>>(v, L, total);
        ANOVA_CHECK_LAUNCH();
        return ANOVA_OK;
    }
    const int64_t nt = (L + kScanTile - 1) / kScanTile;
    if (nt > INT32_MAX) {
        set_error("binning: histogram too long");
        return ANOVA_EINVAL;
    }
    int32_t* tsum = nullptr;
    ANOVA_CUDA_TRY(scratch.alloc(&tsum, nt * sizeof(int32_t)));
    k_scan_tile_sums<<<(unsigned)nt, kScanThreads, 0, st>>>(v, L, tsum);
    k_scan_exclusive<<<1, 1024, 0, st>>>(tsum, nt, total);
    k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, st>>>(v, L, tsum);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// stable scatter: one warp per chunk, ranks of equal bins via match_any
template <typename T>
__global__ void k_bin_scatter(const double* __restrict__ xw, int64_t N, int dA, FrameArgs fr,
                              int nos, int T_, int nb, int nbins, int nchunk,
                              const int32_t* __restrict__ off, int32_t* __restrict__ perm,
                              int32_t* __restrict__ cellout, double* __restrict__ frac64,
                              float* __restrict__ frac32) {
    extern __shared__ int32_t cursor[];
    for (int i = threadIdx.x; i < nbins; i += 32) cursor[i] = off[(int64_t)i * nchunk + blockIdx.x];
    __syncwarp();
    int64_t lo = (int64_t)blockIdx.x * kBinChunk, hi = min(N, lo + kBinChunk);
    const unsigned lane = threadIdx.x;
    for (int64_t base = lo; base < hi; base += 32) {
        int64_t i = base + lane;
        bool valid = i < hi;
        int cell[3] = {0, 0, 0};
        double frac[3] = {0, 0, 0};
        int bin = -1 - (int)lane;  // distinct dummy keys for inactive lanes
        if (valid) {
            node_cell(xw + i * dA, dA, fr.c, fr.s, nos, cell, frac);
            bin = bin_of(cell, dA, T_, nb);
        }
        unsigned peers = __match_any_sync(0xffffffffu, bin);
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        int basepos = 0;
        if (valid && (int)lane == leader) basepos = cursor[bin];
        basepos = __shfl_sync(0xffffffffu, basepos, leader);
        __syncwarp();
        if (valid && (int)lane == leader) cursor[bin] = basepos + __popc(peers);
        __syncwarp();
        if (valid) {
            int64_t pos = basepos + rank;
            perm[pos] = (int32_t)i;
            for (int t = 0; t < dA; t++) {
                cellout[t * N + pos] = cell[t];
                if (frac64) frac64[t * N + pos] = frac[t];
                if (frac32) frac32[t * N + pos] = (float)frac[t];
            }
        }
    }
}

// bin offsets from the scanned per-chunk histogram: bin_start[b] = off[b * nchunk]
__global__ void k_bin_starts(const int32_t* __restrict__ off, int nbins, int nchunk, int64_t N,
                             int32_t* __restrict__ bin_start, int32_t* __restrict__ nchunks_of_bin) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nbins; b += gridDim.x * blockDim.x) {
        int32_t s = (b < nbins) ? off[(int64_t)b * nchunk] : (int32_t)N;
        bin_start[b] = s;
        if (b < nbins) {
            int32_t e = (b + 1 < nbins) ? off[(int64_t)(b + 1) * nchunk] : (int32_t)N;
            nchunks_of_bin[b] = (e - s + kSubChunk - 1) / kSubChunk;
        }
    }
}

__global__ void k_sub_list(const int32_t* __restrict__ bin_start, const int32_t* __restrict__ sub_off,
                           int nbins, int4* __restrict__ sub) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        int32_t s = bin_start[b], e = bin_start[b + 1];
        int32_t k = sub_off[b];
        for (int32_t f = s; f < e; f += kSubChunk) sub[k++] = make_int4(b, f, min(kSubChunk, e - f), 0);
    }
}

// Point sets are allocated from the stream-ordered pool (build_pointset), so
// they go back to it with cudaFreeAsync (cudaFree would not return them).
// Stream-ordered release, no device-wide synchronisation:
void free_pointset_async(PointSet& ps, cudaStream_t st) {
    void* p[6] = {ps.perm, ps.cell, ps.frac64, ps.frac32, ps.bin_start, ps.sub};
    for (void* q : p)
        if (q) cudaFreeAsync(q, st);
    ps = PointSet();
}

// release that has completed on return (owners that free synchronously)
void free_pointset(PointSet& ps) {
    const bool any = ps.perm || ps.cell || ps.frac64 || ps.frac32 || ps.bin_start || ps.sub;
    free_pointset_async(ps, nullptr);
    if (any) cudaStreamSynchronize(nullptr);
}

// ------------------------------------------------------ device allocation
static std::atomic<int64_t> g_fail_countdown{0};   // > 0: allocations left before the one that fails

static bool injected_failure() {
    int64_t v = g_fail_countdown.load();
    while (v > 0)
        if (g_fail_countdown.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
    if (injected_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

// Stream-ordered scratch comes from the device's default pool.  With that pool's
// default release threshold (0) every synchronisation hands its unused memory
// back to the driver, and the next call's allocations map fresh pages (about
// 0.1 ms per call of the window construction).  The library raises the
// threshold once per device to keep up to kPoolKeep bytes of freed scratch
// reserved (never lowering a threshold the application set).
constexpr uint64_t kPoolKeep = (uint64_t)1 << 30;
static std::atomic<uint64_t> g_pool_set{0};        // bit k: device k's pool configured

static void keep_pool_reserve() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    const uint64_t bit = (uint64_t)1 << dev;
    if (g_pool_set.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) == cudaSuccess && thr < kPoolKeep) {
        uint64_t keep = kPoolKeep;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pool_set.fetch_or(bit);
}

cudaError_t dev_malloc_async(void** ptr, size_t bytes, cudaStream_t st) {
    if (injected_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    keep_pool_reserve();
    return cudaMallocAsync(ptr, bytes, st);
}

// Bin and sort the nodes of one window.  coords: device N x dA (user units).
static anova_status build_pointset_impl(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                                        const double* centre, double scale, PointSet& ps, cudaStream_t st);

// On failure the point set is left empty (nothing of it stays allocated).
anova_status build_pointset(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                            int64_t /*ldc*/, const double* centre, double scale, PointSet& ps,
                            cudaStream_t st) {
    free_pointset(ps);
    const anova_status s = build_pointset_impl(plan, w, coords, N, centre, scale, ps, st);
    if (s != ANOVA_OK) free_pointset_async(ps, st);
    return s;
}

static anova_status build_pointset_impl(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                                        const double* centre, double scale, PointSet& ps, cudaStream_t st) {
    ps.N = N;
    const int dA = w.dA;
    const bool want64 = (plan->precision & ANOVA_FP64) != 0;
    const bool want32 = (plan->precision & ANOVA_FP32) != 0;
    if (N == 0) {
        ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.bin_start, (w.nbins + 1) * sizeof(int32_t), st));
        ANOVA_CUDA_TRY(cudaMemsetAsync(ps.bin_start, 0, (w.nbins + 1) * sizeof(int32_t), st));
        return ANOVA_OK;
    }
    ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.perm, N * sizeof(int32_t), st));
    ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.cell, N * dA * sizeof(int32_t), st));
    if (want64) ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.frac64, N * dA * sizeof(double), st));
    if (want32) ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.frac32, N * dA * sizeof(float), st));
    ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.bin_start, (w.nbins + 1) * sizeof(int32_t), st));

    const int nchunk = (int)((N + kBinChunk - 1) / kBinChunk);
    const int64_t L = (int64_t)w.nbins * nchunk;
    int32_t *hist = nullptr, *nch = nullptr, *tot = nullptr;
    Scratch scratch(st);
    ANOVA_CUDA_TRY(scratch.alloc(&hist, L * sizeof(int32_t)));
    ANOVA_CUDA_TRY(scratch.alloc(&nch, (w.nbins + 1) * sizeof(int32_t)));
    ANOVA_CUDA_TRY(scratch.alloc(&tot, 2 * sizeof(int32_t)));
    FrameArgs fr;
    for (int t = 0; t < 3; t++) fr.c[t] = centre[t];
    fr.s = scale;
    const size_t shb = w.nbins * sizeof(int32_t);
    static bool attrs = [] {
        cudaFuncSetAttribute(k_bin_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins * 4);
        cudaFuncSetAttribute(k_bin_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins * 4);
        return true;
    }();
    (void)attrs;
    k_bin_hist<<<nchunk, kThreads, shb, st>>>(coords, N, dA, fr, w.nos, w.T, w.nb, w.nbins, nchunk, hist);
    ANOVA_CHECK_LAUNCH();
    ANOVA_TRY(scan_exclusive(hist, L, tot, scratch, st));
    k_bin_scatter<double><<<nchunk, 32, shb, st>>>(coords, N, dA, fr, w.nos, w.T, w.nb, w.nbins, nchunk,
                                                  hist, ps.perm, ps.cell, ps.frac64, ps.frac32);
    k_bin_starts<<<grid_for(w.nbins + 1, kThreads, 1024), kThreads, 0, st>>>(hist, w.nbins, nchunk, N,
                                                                              ps.bin_start, nch);
    ANOVA_CHECK_LAUNCH();
    ANOVA_TRY(scan_exclusive(nch, w.nbins, tot + 1, scratch, st));
    int32_t totals[2] = {0, 0};
    ANOVA_CUDA_TRY(cudaMemcpyAsync(totals, tot, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    ps.nsub = totals[1];
    if (totals[0] != N) {
        set_error("binning lost nodes");
        return ANOVA_ECUDA;
    }
    ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&ps.sub, std::max(ps.nsub, 1) * sizeof(int4), st));
    k_sub_list<<<grid_for(w.nbins, kThreads, 1024), kThreads, 0, st>>>(ps.bin_start, nch, w.nbins, ps.sub);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// ===================================================================== A2
// Regularised kernel K_R(r) (Sec. 4.2): Gaussian for r <= a = 1/2 - eps_B,
// two-point Taylor polynomial of degree 2p-1 on (a, 1/2] ending at the
// constant c = K(1/2) with vanishing derivatives, c beyond 1/2.
__device__ double gauss_dj(int j, double r, double ell) {
    // d^j/dr^j exp(-(r/ell)^2) = (-1/ell)^j H_j(r/ell) exp(-(r/ell)^2)
    double x = r / ell;
    double h0 = 1.0, h1 = 2.0 * x, hj = (j == 0) ? h0 : h1;
    for (int i = 1; i < j; i++) {
        double h2 = 2.0 * x * h1 - 2.0 * i * h0;
        h0 = h1;
        h1 = h2;
        hj = h2;
    }
    double sc = 1.0;
    for (int i = 0; i < j; i++) sc *= -1.0 / ell;
    return sc * hj * exp(-x * x);
}

__device__ double kreg_dev(double r, double ell, double epsB, int p) {
    const double a = 0.5 - epsB, e = 0.5;
    const double c = exp(-0.25 / (ell * ell));
    if (r <= a) return exp(-(r * r) / (ell * ell));
    if (r > e) return c;
    // Hermite basis on [a, e] with u = (r-a)/(e-a), v = 1-u:
    //   P(r) = sum_j [f^(j)(a) (r-a)^j/j! v^p S_j(u) + f^(j)(e) (r-e)^j/j! u^p S_j(v)],
    //   S_j(z) = sum_{q=0}^{p-1-j} binom(p-1+q, q) z^q.
    const double L = e - a, u = (r - a) / L, v = (e - r) / L;
    double up = 1.0, vp = 1.0;
    for (int i = 0; i < p; i++) { up *= u; vp *= v; }
    double res = 0.0, jfact = 1.0, dra = 1.0;
    for (int j = 0; j < p; j++) {
        if (j > 0) { jfact *= j; dra *= (r - a); }
        double S = 0.0, zq = 1.0, bq = 1.0;  // bq = binom(p-1+q, q)
        for (int q = 0; q <= p - 1 - j; q++) {
            S += bq * zq;
            zq *= u;
            bq = bq * (double)(p + q) / (double)(q + 1);
        }
        res += gauss_dj(j, a, ell) * dra / jfact * vp * S;
    }
    // the end point carries only the value c (its derivatives vanish)
    double S0 = 0.0, zq = 1.0, bq = 1.0;
    for (int q = 0; q <= p - 1; q++) {
        S0 += bq * zq;
        zq *= v;
        bq = bq * (double)(p + q) / (double)(q + 1);
    }
    res += c * up * S0;
    return res;
}

// f[idx] = K_R(||j|| / n), j in I_n^dA (centred index, last axis fastest)
__global__ void k_sample_kreg(int dA, int n, double ell, double epsB, int p, double* __restrict__ f) {
    int64_t tot = 1;
    for (int t = 0; t < dA; t++) tot *= n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = idx;
        double r2 = 0.0;
        for (int t = 0; t < dA; t++) {
            int j = (int)(rem % n) - n / 2;
            rem /= n;
            double v = (double)j / (double)n;
            r2 += v * v;
        }
        f[idx] = kreg_dev(sqrt(r2), ell, epsB, p);
    }
}

// One axis of the real cosine DFT of an even array (shape outer x n x inner):
//   out[k] = sum_j in[j] cos(2 pi k j / n)   (the sine part cancels by symmetry)
__global__ void k_cos_dft_axis(const double* __restrict__ in, double* __restrict__ out, int64_t outer,
                               int n, int64_t inner) {
    int64_t tot = outer * n * inner;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = idx % inner;
        int64_t o = (idx / inner) % n;
        int64_t o0 = idx / (inner * n);
        int k = (int)o - n / 2;
        double acc = 0.0;
        for (int i = 0; i < n; i++) {
            int j = i - n / 2;
            int r = (k * j) % n;
            if (r < 0) r += n;
            acc += in[(o0 * n + i) * inner + s] * cospi(2.0 * (double)r / (double)n);
        }
        out[idx] = acc;
    }
}

// D_k = b_k / prod_t psihat(k_t)^2, psihat = I0(m sqrt(b^2 - (2 pi k/nos)^2)) / phi(0),
// phi(0) = sinh(b m) / (pi m): the transform of the window normalised to psi(0) = 1.
__global__ void k_deconvolve(const double* __restrict__ f, int dA, int n, int nos, int m, double b,
                             double* __restrict__ D64, float* __restrict__ D32) {
    int64_t tot = 1;
    for (int t = 0; t < dA; t++) tot *= n;
    const double phi0 = sinh(b * m) / (M_PI * m);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = idx;
        double den = 1.0;
        for (int t = 0; t < dA; t++) {
            int k = (int)(rem % n) - n / 2;
            rem /= n;
            double w = 2.0 * M_PI * (double)k / (double)nos;
            double ph = cyl_bessel_i0((double)m * sqrt(b * b - w * w)) / phi0;
            den *= ph * ph;
        }
        double v = f[idx] / (double)tot / den;
        if (D64) D64[idx] = v;
        if (D32) D32[idx] = (float)v;
    }
}

// Per-interval polynomials of the normalised window for the FP32 kernels:
// on t in [q - m, q - m + 1), psi(t) is interpolated at kPsiDeg+1 Chebyshev
// points in f = t - (q - m) and rewritten in powers of u = f - 1/2 (FP64),
// kept in FP32 (out, followed by psi(m), the value at the closed end of the
// support) and FP64 (out64).  The interpolation error is below 1.3e-9 of the
// peak at m = 6, sigma = 2 (the window is analytic on each interval).
__global__ void k_psi_poly_fit(int m, double b, double norm, float* __restrict__ out, double* __restrict__ out64) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * m) return;
    constexpr int D = kPsiDeg, K = kPsiDeg + 1;
    double val[K], cheb[K];
    for (int k = 0; k < K; k++) {
        const double f = 0.5 + 0.5 * cospi((k + 0.5) / K);
        const double t = (double)(q - m) + f;
        const double s2 = (double)m * m - t * t;
        double v = 0.0;
        if (s2 > 0.0) {
            const double s = sqrt(s2);
            v = norm * sinh(b * s) / s;
        } else if (s2 == 0.0) {
            v = norm * b;
        }
        val[k] = v;
    }
    for (int i = 0; i < K; i++) {       // Chebyshev coefficients in x = 2u
        double a = 0.0;
        for (int k = 0; k < K; k++) a += val[k] * cospi(i * (k + 0.5) / K);
        cheb[i] = a * 2.0 / K;
    }
    cheb[0] *= 0.5;
    // sum_i cheb_i T_i(x) in powers of x, via T_{i+1} = 2x T_i - T_{i-1}
    double mono[K], tm[K], tc[K], tn[K];
    for (int k = 0; k < K; k++) { mono[k] = 0.0; tm[k] = 0.0; tc[k] = 0.0; }
    tm[0] = 1.0;                        // T_0
    tc[1] = 1.0;                        // T_1
    mono[0] += cheb[0];
    if (D >= 1) mono[1] += cheb[1];
    for (int i = 2; i <= D; i++) {
        for (int k = 0; k < K; k++) tn[k] = -tm[k] + ((k > 0) ? 2.0 * tc[k - 1] : 0.0);
        for (int k = 0; k < K; k++) {
            mono[k] += cheb[i] * tn[k];
            tm[k] = tc[k];
            tc[k] = tn[k];
        }
    }
    double sc = 1.0;                    // x^k = 2^k u^k
    for (int k = 0; k < K; k++) {
        out[q * kPsiStride + k] = (float)(mono[k] * sc);
        out64[q * kPsiStride + k] = mono[k] * sc;
        sc *= 2.0;
    }
    if (q == 0) out[2 * m * kPsiStride] = (float)(norm * b);   // psi(m), the end of the support
}

// exp(-2 pi i r / nos)
__global__ void k_twiddles(int nos, double2* __restrict__ tw64, float2* __restrict__ tw32) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nos; r += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)r / (double)nos, &s, &c);
        if (tw64) tw64[r] = make_double2(c, -s);
        if (tw32) tw32[r] = make_float2((float)c, (float)-s);
    }
}

// ================================================================ set-up
// a requested bin side for the dense kernels: even, region Tb + 2m <= 16, the
// bins within kMaxBins, and the region cells bin Tb - m + r inside [-nos, 2 nos)
// (the kernels wrap an index with one conditional): Tb + m - 2 < nos
static bool dense_side_ok(const WindowPlan& w, int m, int Tb) {
    if (Tb < 2 || Tb % 2 || Tb + 2 * m > 16 || Tb > w.nos) return false;
    if (!(Tb + m - 2 < w.nos)) return false;
    const int64_t nb = (w.nos + Tb - 1) / Tb;
    int64_t nbins = 1;
    for (int t = 0; t < w.dA; t++) nbins *= nb;
    return nbins <= kMaxBins;
}

static void choose_bins(WindowPlan& w, int m, const int* side) {
    if (side && side[w.dA - 1] > 0 && dense_side_ok(w, m, side[w.dA - 1])) {
        const int Tb = side[w.dA - 1];
        const int nb = (w.nos + Tb - 1) / Tb;
        w.dense = true;
        w.T = Tb;
        w.nb = nb;
        w.nbins = nb;
        for (int t = 1; t < w.dA; t++) w.nbins *= nb;
        w.R = Tb + 2 * m;
        return;
    }
    if (w.dA <= 2 && 2 * m + 2 <= 16) {
        // dense small-region kernels: 2-D bins of 2x2 cells (R = 2m + 2); 1-D bins of 16 - 2m cells
        // (R = 16) when the region cells bin*Tb - m + r stay inside [-nos, 2 nos), else 2 cells
        int Tb = 2;
        if (w.dA == 1 && (16 - 2 * m) + m - 2 < w.nos) Tb = 16 - 2 * m;
        const int nb = (w.nos + Tb - 1) / Tb;
        const int nbins = (w.dA == 2) ? nb * nb : nb;
        if (nbins <= kMaxBins) {
            w.dense = true;
            w.T = Tb;
            w.nb = nb;
            w.nbins = nbins;
            w.R = Tb + 2 * m;
            return;
        }
    }
    if (w.dA == 3) {
        // dense tensor-product kernels: bins of Tb^3 cells, region Tb + 2m <= 16
        for (int Tb = 2; Tb <= 4; Tb += 2) {
            const int nb = (w.nos + Tb - 1) / Tb;
            if (Tb + 2 * m <= 16 && nb * nb * nb <= kMaxBins) {
                w.dense = true;
                w.T = Tb;
                w.nb = nb;
                w.nbins = nb * nb * nb;
                w.R = Tb + 2 * m;
                return;
            }
        }
    }
    w.dense = false;
    int T = (w.dA == 3) ? 4 : (w.dA == 2) ? 16 : 64;
    T = std::min(T, w.nos);
    auto nbins_of = [&](int t) {
        int nb = (w.nos + t - 1) / t, nbins = 1;
        for (int i = 0; i < w.dA; i++) nbins *= nb;
        return nbins;
    };
    while (nbins_of(T) > kMaxBins && T < w.nos) T++;
    auto region_bytes = [&](int t) {
        int64_t r = t + 2 * m, v = 1;
        for (int i = 0; i < w.dA; i++) v *= r;
        return v * (int64_t)sizeof(double);
    };
    while (T > 1 && region_bytes(T) > 160 * 1024) T--;
    w.T = T;
    w.nb = (w.nos + T - 1) / T;
    w.nbins = nbins_of(T);
    w.R = T + 2 * m;
}

// min / max cell index per axis over the binned nodes (ints: min at 2t, max at 2t+1)
__global__ void k_cell_range(const int32_t* __restrict__ cell, int64_t N, int dA, int* __restrict__ mm) {
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {-1, -1, -1};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < dA; t++) {
            const int c = cell[t * N + i];
            lo[t] = min(lo[t], c);
            hi[t] = max(hi[t], c);
        }
    for (int t = 0; t < dA; t++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[t] = min(lo[t], __shfl_xor_sync(0xffffffffu, lo[t], o));
            hi[t] = max(hi[t], __shfl_xor_sync(0xffffffffu, hi[t], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[2 * t], lo[t]);
            atomicMax(&mm[2 * t + 1], hi[t]);
        }
    }
}

// FP32 weight table of a dense window: for sorted node pos and axis t < dA,
// wtab[(pos*dA + t)*16 + r] = psi(c_t - (bin_t*T - m) - r + f_t) for r < R, 0 for
// R <= r < 16: the node's offset f_t from its FP64 coordinates, psi from the
// per-interval polynomials in FP64 (Horner), rounded once to FP32.  The one
// tap outside the 2m intervals that can be non-zero is t = m exactly (a node
// on a grid point, f = 0), where psi(m) = `edge` (the window's value at the
// end of its support).
__global__ void k_weight_table(const double* __restrict__ xw, const int32_t* __restrict__ perm, int64_t N,
                               int dA, FrameArgs fr, int nos, int Tb, int R, int m,
                               const double* __restrict__ poly, double edge, float* __restrict__ wtab) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * dA;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = idx / dA;
        const int t = (int)(idx % dA);
        const int64_t i = perm[pos];
        const double xt = fr.s * (xw[i * dA + t] - fr.c[t]);
        const double y = (double)nos * xt;
        const double fl = floor(y);
        const double u = (y - fl) - 0.5;
        int c = (int)fl + nos / 2;
        c %= nos;
        if (c < 0) c += nos;
        const int j0 = c - (c / Tb) * Tb + m;
        float* out = wtab + idx * 16;
        for (int r = 0; r < 16; r++) {
            const int q = j0 - r + m;       // tap at j0 - r + f lies in interval q of [-m, m)
            double w = 0.0;
            if (r < R && q >= 0 && q < 2 * m) {
                const double* cq = poly + q * kPsiStride;
                w = cq[kPsiDeg];
                for (int k = kPsiDeg - 1; k >= 0; k--) w = fma(w, u, cq[k]);
            } else if (r < R && q == 2 * m && u == -0.5) {
                w = edge;
            }
            out[r] = (float)w;
        }
    }
}

// FP64 taps of every node of a window, for the FP64 kernels of the plan's
// own nodes: tap[(pos * dA + t) * (2m + 1) + k] = psi(m - k + f_t), the window
// at the node's offset from cell c_t + k - m, in FP64 exactly as the kernels
// evaluate it (kb_psi); computed once per frame instead of in every product.
__global__ void k_tap_table64(const double* __restrict__ frac64, int64_t N, int dA, int m, double b, double norm,
                              double* __restrict__ tap) {
    const int ntap = 2 * m + 1;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * dA;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = idx / dA;
        const int t = (int)(idx % dA);
        const double f = frac64[t * N + pos];
        double* out = tap + idx * ntap;
        for (int k = 0; k < ntap; k++) out[k] = kb_psi<double>((double)(m - k) + f, (double)m, b, norm);
    }
}

// Box of grid cells that spreading writes and gathering reads: the union of
// the regions [bin*T - m, bin*T + T + m) of the occupied bins, per axis.
static anova_status window_box(anova_plan* plan, WindowPlan& w, cudaStream_t st) {
    for (int t = 0; t < 3; t++) {
        w.box_lo[t] = 0;
        w.box_ext[t] = (t < w.dA) ? w.nos : 1;
    }
    if (w.X.N == 0) return ANOVA_OK;
    int* mm = nullptr;
    Scratch scratch(st, false);
    ANOVA_CUDA_TRY(scratch.alloc(&mm, 6 * sizeof(int)));
    int init[6] = {INT32_MAX, -1, INT32_MAX, -1, INT32_MAX, -1};
    ANOVA_CUDA_TRY(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_cell_range<<<grid_for(w.X.N, kThreads, 2 * plan->sm_count), kThreads, 0, st>>>(w.X.cell, w.X.N, w.dA, mm);
    ANOVA_CHECK_LAUNCH();
    int h[6];
    ANOVA_CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    for (int t = 0; t < w.dA; t++) {
        const int blo = h[2 * t] / w.T, bhi = h[2 * t + 1] / w.T;
        const int ext = (bhi - blo + 1) * w.T + 2 * plan->m;
        if (ext >= w.nos) {
            w.box_lo[t] = 0;
            w.box_ext[t] = w.nos;
        } else {
            w.box_lo[t] = blo * w.T - plan->m;
            w.box_ext[t] = ext;
        }
    }
    return ANOVA_OK;
}

// Frame-dependent part of a window: scaled width, multiplier D_k, binned nodes.
static anova_status window_setup(anova_plan* plan, WindowPlan& w, const double* frame,
                                 double* scratch, cudaStream_t st) {
    for (int t = 0; t < 3; t++) w.centre[t] = frame[t];
    w.scale = frame[3];
    w.ell_l = w.scale * plan->ell;
    int64_t tk = 1;
    for (int t = 0; t < w.dA; t++) tk *= w.n;
    const bool want64 = (plan->precision & ANOVA_FP64) != 0;
    const bool want32 = (plan->precision & ANOVA_FP32) != 0;
    if (!w.D64) ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.D64, tk * sizeof(double)));
    if (want32 && !w.D32) ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.D32, tk * sizeof(float)));
    double* fa = scratch;
    double* fb = scratch + tk;
    const int g = grid_for(tk, kThreads, 4096);
    k_sample_kreg<<<g, kThreads, 0, st>>>(w.dA, w.n, w.ell_l, plan->epsB, plan->p, fa);
    for (int t = 0; t < w.dA; t++) {
        int64_t outer = 1, inner = 1;
        for (int i = 0; i < t; i++) outer *= w.n;
        for (int i = t + 1; i < w.dA; i++) inner *= w.n;
        k_cos_dft_axis<<<g, kThreads, 0, st>>>(fa, fb, outer, w.n, inner);
        std::swap(fa, fb);
    }
    k_deconvolve<<<g, kThreads, 0, st>>>(fa, w.dA, w.n, w.nos, plan->m, plan->b, w.D64,
                                         want32 ? w.D32 : nullptr);
    ANOVA_CHECK_LAUNCH();
    (void)want64;
    ANOVA_TRY(build_pointset(plan, w, w.xw, plan->N, w.dA, w.centre, w.scale, w.X, st));
    // 1-D / 2-D windows on the persistent kernels evaluate their weights on the fly and need no table
    const bool table = w.dense && want32 && plan->N > 0 && !(w.dA < 3 && plan->pw12 && tc5_supported(w.R, plan->m));
    if (table) {
        cudaFree(w.wtab);
        w.wtab = nullptr;
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.wtab, plan->N * 16 * w.dA * sizeof(float)));
        FrameArgs fr;
        for (int t = 0; t < 3; t++) fr.c[t] = w.centre[t];
        fr.s = w.scale;
        k_weight_table<<<grid_for(plan->N * w.dA, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            w.xw, w.X.perm, plan->N, w.dA, fr, w.nos, w.T, w.R, plan->m, plan->psi_poly64, plan->psi_norm * plan->b,
            w.wtab);
        ANOVA_CHECK_LAUNCH();
    } else if (w.wtab) {
        cudaFree(w.wtab);
        w.wtab = nullptr;
    }
    cudaFree(w.wtap64);
    w.wtap64 = nullptr;
    if (want64 && plan->N > 0 && w.X.frac64) {
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.wtap64, (size_t)plan->N * w.dA * (2 * plan->m + 1) * sizeof(double)));
        k_tap_table64<<<grid_for(plan->N * w.dA, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            w.X.frac64, plan->N, w.dA, plan->m, plan->b, plan->psi_norm, w.wtap64);
        ANOVA_CHECK_LAUNCH();
    }
    return window_box(plan, w, st);
}

// tag the sub-problems of window slot w and append them to the merged list
__global__ void k_tag_subs(const int4* __restrict__ src, int n, int slot, int4* __restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 v = src[i];
        v.w = slot;
        dst[i] = v;
    }
}

// Merged sub-problem list and per-window descriptors for the batched dense kernels.
static anova_status build_dense_batch(anova_plan* plan, cudaStream_t st) {
    plan->dense_windows.clear();
    plan->dense_groups.clear();
    int total = 0;
    for (int dA = 1; dA <= 3; dA++)          // windows grouped by dimension and region size (one launch each)
        for (int R = 1; R <= 16; R++) {
            const int first = total;
            for (int l = 0; l < plan->P; l++)
                if (plan->win[l].dense && plan->win[l].dA == dA && plan->win[l].R == R && plan->win[l].X.nsub > 0) {
                    plan->dense_windows.push_back(l);
                    total += plan->win[l].X.nsub;
                }
            if (total > first) plan->dense_groups.push_back({dA * 100 + R, first, total - first});
        }
    plan->dense_nsub = total;
    const int nd = (int)plan->dense_windows.size();
    if (nd == 0) return ANOVA_OK;
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->dense_sub, total * sizeof(int4)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->dense_desc, 2 * nd * sizeof(DenseWin)));
    if (plan->precision & ANOVA_FP32)
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->dense_asort, (size_t)nd * plan->N * sizeof(float)));
    std::vector<DenseWin> desc(2 * nd);
    int at = 0;
    for (int k = 0; k < nd; k++) {
        const WindowPlan& w = plan->win[plan->dense_windows[k]];
        k_tag_subs<<<grid_for(w.X.nsub, kThreads, 256), kThreads, 0, st>>>(w.X.sub, w.X.nsub, k,
                                                                          plan->dense_sub + at);
        at += w.X.nsub;
        for (int prec = 0; prec < 2; prec++) {
            DenseWin& d = desc[prec * nd + k];
            d.perm = w.X.perm;
            d.cell = w.X.cell;
            d.frac = prec == 0 ? (const void*)w.X.frac64 : (const void*)w.X.frac32;
            d.wtab = prec == 0 ? nullptr : w.wtab;
            d.wtap = prec == 0 ? w.wtap64 : nullptr;
            d.asort = (prec == 0 || !plan->dense_asort) ? nullptr : plan->dense_asort + (size_t)k * plan->N;
            d.grid = prec == 0 ? (void*)(static_cast<double*>(plan->grid) + w.grid_off)
                               : (void*)(static_cast<float*>(plan->grid) + w.grid_off);
            const int l = plan->dense_windows[k];
            d.out = prec == 0 ? (void*)(static_cast<double*>(plan->tmp) + (int64_t)l * plan->N)
                              : (void*)(static_cast<float*>(plan->tmp) + (int64_t)l * plan->N);
            d.N = w.X.N;
            d.nos = w.nos;
            d.Tb = w.T;
            d.nb = w.nb;
            d.pad = 0;
        }
    }
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->dense_desc, desc.data(), 2 * nd * sizeof(DenseWin),
                                   cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// Descriptors of the 3-D windows that use the batched box FFT.
static anova_status build_fft3_batch(anova_plan* plan, cudaStream_t st) {
    plan->fft3_windows.clear();
    for (int l = 0; l < plan->P; l++)
        if (fft3_box_supported(plan->win[l])) plan->fft3_windows.push_back(l);
    const int nw = (int)plan->fft3_windows.size();
    if (nw == 0) return ANOVA_OK;
    plan->fft3_slab = true;
    for (int l : plan->fft3_windows) plan->fft3_slab = plan->fft3_slab && fft3_slab_supported(plan->win[l]);
    std::vector<Fft3Win> desc(2 * nw);
    for (int k = 0; k < nw; k++) {
        const WindowPlan& w = plan->win[plan->fft3_windows[k]];
        for (int prec = 0; prec < 2; prec++) {
            Fft3Win& d = desc[prec * nw + k];
            if (prec == 0) {
                d.grid = static_cast<double*>(plan->grid) + w.grid_off;
                d.buf1 = static_cast<double2*>(plan->work1) + w.work_off;
                d.buf2 = static_cast<double2*>(plan->work2) + w.work_off;
                d.tw = w.tw64;
                d.D = w.D64;
            } else {
                d.grid = static_cast<float*>(plan->grid) + w.grid_off;
                d.buf1 = static_cast<float2*>(plan->work1) + w.work_off;
                d.buf2 = static_cast<float2*>(plan->work2) + w.work_off;
                d.tw = w.tw32;
                d.D = w.D32;
            }
            for (int t = 0; t < 3; t++) {
                d.lo[t] = w.box_lo[t];
                d.B[t] = w.box_ext[t];
            }
            d.n = w.n;
            d.nos = w.nos;
        }
    }
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->fft3_desc, 2 * nw * sizeof(Fft3Win)));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->fft3_desc, desc.data(), 2 * nw * sizeof(Fft3Win),
                                   cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

// Descriptors of the batched 1-D / 2-D box FFT: every such window whose box
// transform fits one thread block's shared memory in FP64.
static anova_status build_fft12_batch(anova_plan* plan, cudaStream_t st) {
    plan->fft12_windows.clear();
    for (int l = 0; l < plan->P; l++) {
        WindowPlan& w = plan->win[l];
        w.fft12 = plan->N > 0 && fft12_box_supported(w);
        if (w.fft12) plan->fft12_windows.push_back(l);
    }
    const int nw = (int)plan->fft12_windows.size();
    if (nw == 0) return ANOVA_OK;
    std::vector<Fft12Win> desc(2 * nw);
    plan->fft12_smem64 = plan->fft12_smem32 = 0;
    for (int k = 0; k < nw; k++) {
        const WindowPlan& w = plan->win[plan->fft12_windows[k]];
        const int un = w.nos == 2 * w.n ? w.n : 0;
        plan->fft12_uniform_n = (k == 0) ? un : (plan->fft12_uniform_n == un ? un : 0);
        plan->fft12_smem64 = std::max(plan->fft12_smem64, fft12_window_smem(w, sizeof(double)));
        plan->fft12_smem32 = std::max(plan->fft12_smem32, fft12_window_smem(w, sizeof(float)));
        for (int prec = 0; prec < 2; prec++) {
            Fft12Win& d = desc[prec * nw + k];
            d.grid = prec == 0 ? (void*)(static_cast<double*>(plan->grid) + w.grid_off)
                               : (void*)(static_cast<float*>(plan->grid) + w.grid_off);
            d.tw = prec == 0 ? (const void*)w.tw64 : (const void*)w.tw32;
            d.D = prec == 0 ? (const void*)w.D64 : (const void*)w.D32;
            d.dA = w.dA;
            d.n = w.n;
            d.nos = w.nos;
            for (int t = 0; t < 2; t++) {
                d.lo[t] = w.box_lo[t];
                d.B[t] = w.box_ext[t];
            }
        }
    }
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->fft12_desc, 2 * nw * sizeof(Fft12Win)));
    ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->fft12_desc, desc.data(), 2 * nw * sizeof(Fft12Win),
                                   cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    return ANOVA_OK;
}

static anova_status validate(int64_t N, int32_t d, int64_t ld, const int32_t* windows, int32_t P,
                             const double* weights, double ell, const int32_t* n, int32_t m,
                             double sigma, double eps_B, int32_t p, int32_t precision) {
    auto bad = [](const std::string& s) {
        set_error(s);
        return ANOVA_EINVAL;
    };
    if (N < 0 || N > INT32_MAX) return bad("N must be in [0, 2^31)");
    if (d < 1 || ld < d) return bad("need d >= 1 and ld >= d");
    if (!windows || P < 1 || P > kMaxWindows) return bad("need 1 <= P <= 256 windows");
    for (int l = 0; l < P; l++) {
        int dA = 0;
        while (dA < 3 && windows[3 * l + dA] >= 0) dA++;
        if (dA == 0) return bad("empty window " + std::to_string(l));
        for (int t = dA; t < 3; t++)
            if (windows[3 * l + t] != -1) return bad("window padding must be -1 at the end");
        for (int t = 0; t < dA; t++) {
            if (windows[3 * l + t] >= d) return bad("feature index out of range in window " + std::to_string(l));
            for (int u = 0; u < t; u++)
                if (windows[3 * l + t] == windows[3 * l + u]) return bad("repeated feature in a window");
        }
        if (weights && !std::isfinite(weights[l])) return bad("non-finite weight");
        int nl = n ? n[l] : 32;
        if (nl < 4 || (nl & 1)) return bad("n must be even and >= 4");
        double nosd = sigma * nl;
        int nos = (int)std::lround(nosd);
        if (std::fabs(nosd - nos) > 1e-9 || (nos & 1)) return bad("sigma*n must be an even integer");
        if (2 * m + 2 > nos) return bad("need 2m+2 <= sigma*n");
        int64_t big = 1;
        for (int t = 0; t < dA; t++) big *= nos;
        if (big > (int64_t)1 << 24) return bad("grid (sigma*n)^dims above 2^24 cells");
    }
    if (!(ell > 0.0) || !std::isfinite(ell)) return bad("ell must be positive and finite");
    if (m < 1 || m > kMaxM) return bad("m must be in [1, 12]");
    if (!(sigma >= 1.0) || sigma > 8.0) return bad("sigma must be in [1, 8]");
    if (!(eps_B > 0.0 && eps_B < 0.5)) return bad("eps_B must be in (0, 1/2)");
    if (p < 1 || p > 16) return bad("p must be in [1, 16]");
    if (precision < 1 || precision > 3) return bad("precision must be ANOVA_FP64, ANOVA_FP32 or ANOVA_MIXED");
    return ANOVA_OK;
}

static anova_status plan_build(const double* points, int64_t N, int32_t d, int64_t ld,
                               const int32_t* windows, int32_t P, const double* weights, double ell,
                               const int32_t* n, int32_t m, double sigma, double eps_B, int32_t p,
                               int32_t precision, cudaStream_t st, anova_plan* plan) {
    int dev = 0;
    ANOVA_CUDA_TRY(cudaGetDevice(&dev));
    ANOVA_CUDA_TRY(cudaDeviceGetAttribute(&plan->sm_count, cudaDevAttrMultiProcessorCount, dev));
    plan->N = N;
    plan->d = d;
    plan->P = P;
    plan->m = m;
    plan->p = p;
    plan->precision = precision;
    plan->sigma = sigma;
    plan->epsB = eps_B;
    plan->ell = ell;
    plan->b = M_PI * (2.0 - 1.0 / sigma);
    plan->psi_norm = (double)m / std::sinh(plan->b * m);
    {
        int lowest = 0, highest = 0;
        ANOVA_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lowest, &highest));
        ANOVA_CUDA_TRY(cudaStreamCreateWithPriority(&plan->side, cudaStreamNonBlocking, lowest));
        ANOVA_CUDA_TRY(cudaStreamCreateWithPriority(&plan->side_hi, cudaStreamNonBlocking, highest));
        // the 1-D / 2-D chain forked before the 3-D spread and queued after it: the fastest of
        // the schedules on the precision form (0.952 ms against 0.961 ms queued first, 0.995 ms
        // on one stream)
        plan->overlap12 = 2;
    }
    ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming));
    ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming));
    plan->win.resize(P);
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->psi_poly, (2 * m * kPsiStride + 1) * sizeof(float)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->psi_poly64, 2 * m * kPsiStride * sizeof(double)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->f16_scale, sizeof(unsigned)));
    k_psi_poly_fit<<<1, 64, 0, st>>>(m, plan->b, plan->psi_norm, plan->psi_poly, plan->psi_poly64);
    ANOVA_CHECK_LAUNCH();
    plan->psi_host.assign(2 * m * kPsiStride, 0.f);
    ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->psi_host.data(), plan->psi_poly, plan->psi_host.size() * sizeof(float),
                                   cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    size_t max_tk = 1;
    for (int l = 0; l < P; l++) {
        WindowPlan& w = plan->win[l];
        w.dA = 0;
        while (w.dA < 3 && windows[3 * l + w.dA] >= 0) {
            w.feat[w.dA] = windows[3 * l + w.dA];
            w.dA++;
        }
        w.n = n ? n[l] : 32;
        w.nos = (int)std::lround(sigma * w.n);
        w.eta = weights ? weights[l] : 1.0 / P;
        choose_bins(w, m, plan->bin_side);
        if (w.nbins > kMaxBins) {
            set_error("window " + std::to_string(l) + ": grid too fine for the binning (reduce n or m)");
            return ANOVA_EINVAL;
        }
        size_t ge = 1, we = w.n, tk = 1;
        for (int t = 0; t < w.dA; t++) { ge *= w.nos; tk *= w.n; }
        for (int t = 1; t < w.dA; t++) we *= w.nos;
        w.grid_off = plan->grid_elems;
        w.work_off = plan->work_elems;
        plan->grid_elems += (ge + 63) / 64 * 64;
        plan->work_elems += (we + 63) / 64 * 64;
        max_tk = std::max(max_tk, tk);
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.tw64, w.nos * sizeof(double2)));
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.tw32, w.nos * sizeof(float2)));
        k_twiddles<<<grid_for(w.nos, kThreads, 64), kThreads, 0, st>>>(w.nos, w.tw64, w.tw32);
        ANOVA_CHECK_LAUNCH();
        if (N > 0) {
            ANOVA_CUDA_TRY(anova::dev_malloc((void**)&w.xw, N * w.dA * sizeof(double)));
            k_extract<<<grid_for(N, kThreads, 4 * plan->sm_count), kThreads, 0, st>>>(
                points, N, ld, w.dA, w.feat[0], w.feat[1], w.feat[2], w.xw);
            ANOVA_CHECK_LAUNCH();
        }
    }
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->grid, plan->grid_elems * sizeof(double)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->work1, plan->work_elems * sizeof(double2)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->work2, plan->work_elems * sizeof(double2)));
    ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->tmp, std::max<int64_t>(N, 1) * P * sizeof(double)));
    {
        std::vector<double> eta(P);
        for (int l = 0; l < P; l++) eta[l] = plan->win[l].eta;
        ANOVA_CUDA_TRY(anova::dev_malloc((void**)&plan->eta_dev, P * sizeof(double)));
        ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->eta_dev, eta.data(), P * sizeof(double),
                                       cudaMemcpyHostToDevice, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // scratch for frames and D_k set-up
    const int nblk = grid_for(std::max<int64_t>(N, 1), kThreads, 2 * plan->sm_count);
    size_t scratch_elems = std::max<size_t>(6 * nblk + 8, 2 * max_tk);
    double* scratch = nullptr;
    Scratch guard(st, false);
    ANOVA_CUDA_TRY(guard.alloc(&scratch, scratch_elems * sizeof(double)));
    anova_status s = ANOVA_OK;
    for (int l = 0; l < P && s == ANOVA_OK; l++) {
        WindowPlan& w = plan->win[l];
        double frame[5] = {0, 0, 0, 1.0, 0};
        if (N > 0) s = compute_frame(plan, w.xw, N, nullptr, 0, w.dA, scratch, frame, st);
        if (s == ANOVA_OK) s = window_setup(plan, w, frame, scratch, st);
    }
    if (s == ANOVA_OK) s = build_dense_batch(plan, st);
    if (s == ANOVA_OK) s = build_fft3_batch(plan, st);
    if (s == ANOVA_OK) s = build_fft12_batch(plan, st);
    if (s == ANOVA_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("plan: ") + cudaGetErrorString(e));
            s = ANOVA_ECUDA;
        }
    }
    return s;
}

// Rebuild window l of `dst` (a copy of the plan's window) in the frame spanned by
// the training nodes and the extra coordinates zw (M x dA), for predictions
// outside the plan's ball.
anova_status window_reframe(anova_plan* plan, int l, const double* zw, int64_t M, WindowPlan& dst,
                            cudaStream_t st) {
    const WindowPlan& src = plan->win[l];
    dst = WindowPlan();
    dst.dA = src.dA;
    for (int t = 0; t < 3; t++) dst.feat[t] = src.feat[t];
    dst.n = src.n;
    dst.nos = src.nos;
    dst.T = src.T;
    dst.nb = src.nb;
    dst.R = src.R;
    dst.nbins = src.nbins;
    dst.dense = src.dense;
    dst.grid_off = src.grid_off;
    dst.work_off = src.work_off;
    dst.eta = src.eta;
    dst.tw64 = src.tw64;   // borrowed
    dst.tw32 = src.tw32;   // borrowed
    dst.xw = src.xw;       // borrowed
    int64_t tk = 1;
    for (int t = 0; t < src.dA; t++) tk *= src.n;
    const int nblk = grid_for(plan->N + M, kThreads, 2 * plan->sm_count);
    double* scratch = nullptr;
    Scratch guard(st, false);
    ANOVA_CUDA_TRY(guard.alloc(&scratch, std::max<size_t>(6 * nblk + 8, 2 * tk) * sizeof(double)));
    double frame[5];
    anova_status s = compute_frame(plan, src.xw, plan->N, zw, M, src.dA, scratch, frame, st);
    if (s == ANOVA_OK) s = window_setup(plan, dst, frame, scratch, st);
    cudaStreamSynchronize(st);
    return s;
}

// Window l in the frame of the plan's own, with the same centre and the scale
// divided by rho >= 1: every point within rho times the nodes' radius of the
// centre maps into the ball.  Same buffers as window_reframe.
anova_status window_widened(anova_plan* plan, int l, double rho, WindowPlan& dst, cudaStream_t st) {
    const WindowPlan& src = plan->win[l];
    dst = WindowPlan();
    dst.dA = src.dA;
    for (int t = 0; t < 3; t++) dst.feat[t] = src.feat[t];
    dst.n = src.n;
    dst.nos = src.nos;
    dst.T = src.T;
    dst.nb = src.nb;
    dst.R = src.R;
    dst.nbins = src.nbins;
    dst.dense = src.dense;
    dst.grid_off = src.grid_off;
    dst.work_off = src.work_off;
    dst.eta = src.eta;
    dst.tw64 = src.tw64;   // borrowed
    dst.tw32 = src.tw32;   // borrowed
    dst.xw = src.xw;       // borrowed
    int64_t tk = 1;
    for (int t = 0; t < src.dA; t++) tk *= src.n;
    double* scratch = nullptr;
    Scratch guard(st, false);
    ANOVA_CUDA_TRY(guard.alloc(&scratch, std::max<size_t>(16, 2 * tk) * sizeof(double)));
    const double frame[5] = {src.centre[0], src.centre[1], src.centre[2], src.scale / rho, 0.0};
    anova_status s = window_setup(plan, dst, frame, scratch, st);
    cudaStreamSynchronize(st);
    return s;
}

void window_release_reframed(WindowPlan& w) {
    cudaFree(w.wtab);
    cudaFree(w.wtap64);
    cudaFree(w.D64);
    cudaFree(w.D32);
    free_pointset(w.X);
    w = WindowPlan();
}

// max ||z - centre|| over M coordinates (device M x dA)
anova_status max_radius(anova_plan* plan, const double* zw, int64_t M, int dA, const double* centre,
                        double* rmax_host, cudaStream_t st) {
    *rmax_host = 0.0;
    if (M == 0) return ANOVA_OK;
    const int nblk = grid_for(M, kThreads, 2 * plan->sm_count);
    double* scratch = nullptr;
    Scratch guard(st);
    ANOVA_CUDA_TRY(guard.alloc(&scratch, (nblk + 8) * sizeof(double)));
    double* frame = scratch + nblk;
    double hf[5] = {centre[0], centre[1], centre[2], 1.0, 0.0};
    ANOVA_CUDA_TRY(cudaMemcpyAsync(frame, hf, 5 * sizeof(double), cudaMemcpyHostToDevice, st));
    k_maxnorm<<<nblk, kThreads, 0, st>>>(zw, M, nullptr, 0, dA, frame, scratch);
    k_maxnorm_final<<<1, kThreads, 0, st>>>(scratch, nblk, 1.0, frame);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemcpyAsync(hf, frame, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    *rmax_host = hf[4];
    return ANOVA_OK;
}

// ---------------------------------------------------------------------------
// Variants of the binning and radius helpers that write into caller-provided
// device buffers instead of allocating (used by krr_predict_noalloc).
NoallocBinBuffers noalloc_bin_layout(int64_t M) {
    NoallocBinBuffers b;
    b.nchunk = (int)((M + kBinChunk - 1) / kBinChunk);
    b.hist_elems = (int64_t)kMaxBins * std::max(b.nchunk, 1);
    b.sub_capacity = kMaxBins + (int)(M / kSubChunk) + 1;
    b.red_elems = 6 * 2 * 1024 + 16;
    return b;
}

anova_status max_radius_into(anova_plan* plan, const double* zw, int64_t M, int dA, const double* centre,
                             double* red, double* rmax_host, cudaStream_t st) {
    *rmax_host = 0.0;
    if (M == 0) return ANOVA_OK;
    const int nblk = grid_for(M, kThreads, std::min(2 * plan->sm_count, 2048));
    double* frame = red + nblk;
    double hf[5] = {centre[0], centre[1], centre[2], 1.0, 0.0};
    ANOVA_CUDA_TRY(cudaMemcpyAsync(frame, hf, 5 * sizeof(double), cudaMemcpyHostToDevice, st));
    k_maxnorm<<<nblk, kThreads, 0, st>>>(zw, M, nullptr, 0, dA, frame, red);
    k_maxnorm_final<<<1, kThreads, 0, st>>>(red, nblk, 1.0, frame);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemcpyAsync(hf, frame, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    *rmax_host = hf[4];
    return ANOVA_OK;
}

anova_status build_pointset_into(anova_plan* plan, WindowPlan& w, const double* coords, int64_t N,
                                 const double* centre, double scale, const NoallocBinBuffers& buf,
                                 PointSet& ps, cudaStream_t st) {
    ps.N = N;
    ps.perm = buf.perm;
    ps.cell = buf.cell;
    ps.frac64 = (plan->precision & ANOVA_FP64) ? buf.frac64 : nullptr;
    ps.frac32 = (plan->precision & ANOVA_FP32) ? buf.frac32 : nullptr;
    ps.bin_start = buf.bin_start;
    ps.sub = buf.sub;
    ps.nsub = 0;
    if (N == 0) return ANOVA_OK;
    const int dA = w.dA;
    const int nchunk = (int)((N + kBinChunk - 1) / kBinChunk);
    const int64_t L = (int64_t)w.nbins * nchunk;
    if (nchunk > buf.nchunk || L > buf.hist_elems) {
        set_error("no-alloc binning: scratch too small");
        return ANOVA_EINVAL;
    }
    FrameArgs fr;
    for (int t = 0; t < 3; t++) fr.c[t] = centre[t];
    fr.s = scale;
    const size_t shb = w.nbins * sizeof(int32_t);
    static bool attrs = [] {
        cudaFuncSetAttribute(k_bin_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins * 4);
        cudaFuncSetAttribute(k_bin_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins * 4);
        return true;
    }();
    (void)attrs;
    k_bin_hist<<<nchunk, kThreads, shb, st>>>(coords, N, dA, fr, w.nos, w.T, w.nb, w.nbins, nchunk, buf.hist);
    k_scan_exclusive<<<1, 1024, 0, st>>>(buf.hist, L, buf.tot);
    k_bin_scatter<double><<<nchunk, 32, shb, st>>>(coords, N, dA, fr, w.nos, w.T, w.nb, w.nbins, nchunk,
                                                  buf.hist, ps.perm, ps.cell, ps.frac64, ps.frac32);
    k_bin_starts<<<grid_for(w.nbins + 1, kThreads, 1024), kThreads, 0, st>>>(buf.hist, w.nbins, nchunk, N,
                                                                              ps.bin_start, buf.nch);
    k_scan_exclusive<<<1, 1024, 0, st>>>(buf.nch, w.nbins, buf.tot + 1);
    ANOVA_CHECK_LAUNCH();
    int32_t totals[2] = {0, 0};
    ANOVA_CUDA_TRY(cudaMemcpyAsync(totals, buf.tot, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (totals[0] != N) {
        set_error("no-alloc binning lost nodes");
        return ANOVA_ECUDA;
    }
    if (totals[1] > buf.sub_capacity) {
        set_error("no-alloc binning: too many sub-problems for the scratch");
        return ANOVA_EINVAL;
    }
    ps.nsub = totals[1];
    k_sub_list<<<grid_for(w.nbins, kThreads, 1024), kThreads, 0, st>>>(ps.bin_start, buf.nch, w.nbins, ps.sub);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// copy the window's feature columns of Z into zw (M x dA)
anova_status extract_window(anova_plan* plan, const double* Z, int64_t M, int64_t ldz, const WindowPlan& w,
                            double* zw, cudaStream_t st) {
    if (M == 0) return ANOVA_OK;
    k_extract<<<grid_for(M, kThreads, 4 * plan->sm_count), kThreads, 0, st>>>(
        Z, M, ldz, w.dA, w.feat[0], w.feat[1], w.feat[2], zw);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

}  // namespace anova

using namespace anova;

extern "C" {

anova_status anova_fastsum_plan(const double* points, int64_t N, int32_t d, int64_t ld,
                                const int32_t* windows, int32_t P, const double* weights,
                                double ell, const int32_t* n, int32_t m, double sigma,
                                double eps_B, int32_t p, int32_t precision, void* stream,
                                anova_plan** out) {
    return anova_fastsum_plan_bins(points, N, d, ld, windows, P, weights, ell, n, m, sigma, eps_B, p, precision,
                                   nullptr, stream, out);
}

anova_status anova_fastsum_plan_bins(const double* points, int64_t N, int32_t d, int64_t ld,
                                     const int32_t* windows, int32_t P, const double* weights, double ell,
                                     const int32_t* n, int32_t m, double sigma, double eps_B, int32_t p,
                                     int32_t precision, const int32_t* bin_side, void* stream, anova_plan** out) {
    set_error("");
    if (!out) {
        set_error("out is NULL");
        return ANOVA_EINVAL;
    }
    *out = nullptr;
    if (N > 0 && !points) {
        set_error("points is NULL");
        return ANOVA_EINVAL;
    }
    ANOVA_TRY(validate(N, d, ld, windows, P, weights, ell, n, m, sigma, eps_B, p, precision));
    anova_plan* plan = new (std::nothrow) anova_plan();
    if (!plan) return ANOVA_ENOMEM;
    if (bin_side)
        for (int t = 0; t < 3; t++) plan->bin_side[t] = bin_side[t] > 0 ? bin_side[t] : 0;
    anova_status s = plan_build(points, N, d, ld, windows, P, weights, ell, n, m, sigma, eps_B, p,
                                precision, (cudaStream_t)stream, plan);
    if (s != ANOVA_OK) {
        cudaGetLastError();
        anova_plan_destroy(plan);
        return s;
    }
    *out = plan;
    return ANOVA_OK;
}

void anova_plan_destroy(anova_plan* plan) {
    if (!plan) return;
    for (auto& w : plan->win) {
        cudaFree(w.wtab);
        cudaFree(w.wtap64);
        cudaFree(w.D64);
        cudaFree(w.D32);
        cudaFree(w.tw64);
        cudaFree(w.tw32);
        cudaFree(w.xw);
        free_pointset(w.X);
    }
    cudaFree(plan->grid);
    cudaFree(plan->work1);
    cudaFree(plan->work2);
    cudaFree(plan->tmp);
    cudaFree(plan->eta_dev);
    cudaFree(plan->dense_sub);
    cudaFree(plan->dense_desc);
    cudaFree(plan->dense_asort);
    cudaFree(plan->fft3_desc);
    cudaFree(plan->fft12_desc);
    cudaFree(plan->psi_poly);
    cudaFree(plan->psi_poly64);
    cudaFree(plan->f16_scale);
    if (plan->side) cudaStreamDestroy(plan->side);
    if (plan->side_hi) cudaStreamDestroy(plan->side_hi);
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    cudaFree(plan->cg_vec);
    cudaFree(plan->cg_scal);
    cudaFree(plan->cg_part);
    for (auto e : plan->clock.ev) cudaEventDestroy(e);
    for (auto& g : plan->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
    delete plan;
}

anova_status anova_debug_fail_alloc(int64_t k) {
    if (k < 0) {
        anova::set_error("anova_debug_fail_alloc: k must be >= 0");
        return ANOVA_EINVAL;
    }
    g_fail_countdown.store(k);
    return ANOVA_OK;
}

anova_status anova_debug_memory(int64_t* free_bytes, int64_t* pool_used_bytes, int64_t* pool_reserved_bytes) {
    size_t fr = 0, total = 0;
    ANOVA_CUDA_TRY(cudaMemGetInfo(&fr, &total));
    int dev = 0;
    ANOVA_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    ANOVA_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t used = 0;
    ANOVA_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    uint64_t reserved = 0;
    ANOVA_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    if (free_bytes) *free_bytes = (int64_t)fr;
    if (pool_used_bytes) *pool_used_bytes = (int64_t)used;
    if (pool_reserved_bytes) *pool_reserved_bytes = (int64_t)reserved;
    return ANOVA_OK;
}

const char* anova_status_string(anova_status s) {
    switch (s) {
        case ANOVA_OK: return "ANOVA_OK: success";
        case ANOVA_EINVAL: return "ANOVA_EINVAL: invalid argument";
        case ANOVA_ENOMEM: return "ANOVA_ENOMEM: device allocation failed";
        case ANOVA_ECUDA: return "ANOVA_ECUDA: CUDA call failed";
        case ANOVA_ENOCONV: return "ANOVA_ENOCONV: CG reached maxit";
        case ANOVA_ERANGE: return "ANOVA_ERANGE: input out of range";
        case ANOVA_ETIMEOUT: return "ANOVA_ETIMEOUT: device wait expired";
        case ANOVA_EBUSY: return "ANOVA_EBUSY: refused, the expected queue wait exceeds the bound";
    }
    return "unknown anova_status";
}

const char* anova_last_error(void) { return g_last_error.c_str(); }

anova_status anova_plan_window(const anova_plan* plan, int32_t l, double* centre, double* scale,
                               double* ell_l, int32_t* dims, int32_t* n, int32_t* nos) {
    if (!plan || l < 0 || l >= plan->P) {
        set_error("bad plan or window index");
        return ANOVA_EINVAL;
    }
    const WindowPlan& w = plan->win[l];
    if (centre) for (int t = 0; t < 3; t++) centre[t] = w.centre[t];
    if (scale) *scale = w.scale;
    if (ell_l) *ell_l = w.ell_l;
    if (dims) *dims = w.dA;
    if (n) *n = w.n;
    if (nos) *nos = w.nos;
    return ANOVA_OK;
}

anova_status anova_plan_window_bins(const anova_plan* plan, int32_t l, int32_t* bin_side, int32_t* region,
                                    int32_t* dense) {
    if (!plan || l < 0 || l >= plan->P) {
        set_error("bad plan or window index");
        return ANOVA_EINVAL;
    }
    const WindowPlan& w = plan->win[l];
    if (bin_side) *bin_side = w.T;
    if (region) *region = w.R;
    if (dense) *dense = w.dense ? 1 : 0;
    return ANOVA_OK;
}

anova_status anova_plan_bin_rule(int32_t dims, int32_t n, int32_t m, double sigma, const int32_t* bin_side,
                                 int32_t* side, int32_t* region, int32_t* dense, int32_t* nbins) {
    if (dims < 1 || dims > 3) {
        set_error("anova_plan_bin_rule: dims must be 1, 2 or 3");
        return ANOVA_EINVAL;
    }
    const int32_t win[3] = {0, dims > 1 ? 1 : -1, dims > 2 ? 2 : -1};
    ANOVA_TRY(validate(0, dims, dims, win, 1, nullptr, 1.0, &n, m, sigma, 1.0 / 16, 8, ANOVA_FP64));
    WindowPlan w;
    w.dA = dims;
    w.n = n;
    w.nos = (int)std::lround(sigma * n);
    int32_t req[3] = {0, 0, 0};
    if (bin_side)
        for (int t = 0; t < 3; t++) req[t] = bin_side[t] > 0 ? bin_side[t] : 0;
    choose_bins(w, m, req);
    if (side) *side = w.T;
    if (region) *region = w.R;
    if (dense) *dense = w.dense ? 1 : 0;
    if (nbins) *nbins = w.nbins;
    if (w.nbins > kMaxBins) {
        set_error("anova_plan_bin_rule: grid too fine for the binning (reduce n or m)");
        return ANOVA_EINVAL;
    }
    return ANOVA_OK;
}

anova_status anova_debug_diag(const anova_plan* plan, int32_t l, double* D_host) {
    if (!plan || l < 0 || l >= plan->P || !D_host) {
        set_error("bad plan, window index or output");
        return ANOVA_EINVAL;
    }
    const WindowPlan& w = plan->win[l];
    int64_t tk = 1;
    for (int t = 0; t < w.dA; t++) tk *= w.n;
    ANOVA_CUDA_TRY(cudaMemcpy(D_host, w.D64, tk * sizeof(double), cudaMemcpyDeviceToHost));
    return ANOVA_OK;
}

}  // extern "C"
