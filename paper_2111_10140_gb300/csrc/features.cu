// features.cu -- window construction upstream of the fast summation
// (arXiv 2111.10140, Sec. 5: features ranked by mutual information score,
// those below a threshold dropped, the rest grouped three at a time in rank
// order; Sec. 6.1: z-score normalisation with training statistics).
//
// Column statistics read the row-major matrix in coalesced row blocks; each
// block keeps per-column partials in shared memory and the column totals are
// summed over the blocks in a fixed order.  The score is the plug-in mutual
// information between the label and the feature's quantile bin, the quantile
// bins coming from a fine equal-width histogram (bin of a value: floor((v -
// lo) F / (hi - lo)), F = 4096, the last bin closed; quantile bin of fine bin
// j: floor(B (2 C_j + c_j) / (2 N)) with C_j the count below j and c_j its
// own count, in integers).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace anova {

constexpr int kFeatMaxD = 2048;          // columns handled by the statistics kernels
constexpr int kFine = 4096;
constexpr int kStatRows = 256;           // rows per block of the statistics kernels
constexpr int kMaxClasses = 64;
constexpr int kMaxQBins = 64;

// total order of doubles as unsigned integers (for min / max by integer atomics)
__device__ __forceinline__ unsigned long long ord_of(double v) {
    const unsigned long long u = __double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double of_ord(unsigned long long u) {
    return __longlong_as_double((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u);
}

// per block: column sums of x (mode 0) or of (x - mean)^2 (mode 1), and in mode 0 min / max
__global__ void __launch_bounds__(kThreads)
k_col_partials(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ mean, int mode,
               double* __restrict__ psum, unsigned long long* __restrict__ pmin,
               unsigned long long* __restrict__ pmax) {
    extern __shared__ __align__(16) unsigned char sm[];
    double* ssum = reinterpret_cast<double*>(sm);
    unsigned long long* smin = reinterpret_cast<unsigned long long*>(ssum + d);
    unsigned long long* smax = smin + d;
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        ssum[c] = 0.0;
        smin[c] = ~0ull;
        smax[c] = 0ull;
    }
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kStatRows;
    const int64_t rows = (N - r0 < kStatRows) ? (N - r0) : kStatRows;
    for (int64_t e = threadIdx.x; e < rows * d; e += blockDim.x) {
        const int64_t r = r0 + e / d;
        const int c = (int)(e % d);
        const double v = X[r * ld + c];
        if (mode == 0) {
            atomicAdd(&ssum[c], v);
            const unsigned long long o = ord_of(v);
            atomicMin(&smin[c], o);
            atomicMax(&smax[c], o);
        } else {
            const double t = v - mean[c];
            atomicAdd(&ssum[c], t * t);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        psum[(size_t)blockIdx.x * d + c] = ssum[c];
        if (mode == 0) {
            pmin[(size_t)blockIdx.x * d + c] = smin[c];
            pmax[(size_t)blockIdx.x * d + c] = smax[c];
        }
    }
}

// column totals over the blocks (fixed order); mode 0: mean, lo, hi; mode 1: std
__global__ void k_col_totals(const double* __restrict__ psum, const unsigned long long* __restrict__ pmin,
                             const unsigned long long* __restrict__ pmax, int nblk, int d, int64_t N, int mode,
                             double* __restrict__ out0, double* __restrict__ lo, double* __restrict__ hi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int b = 0; b < nblk; b++) {
        s += psum[(size_t)b * d + c];
        if (mode == 0) {
            const unsigned long long a = pmin[(size_t)b * d + c], z = pmax[(size_t)b * d + c];
            mn = a < mn ? a : mn;
            mx = z > mx ? z : mx;
        }
    }
    if (mode == 0) {
        out0[c] = s / (double)N;
        if (lo) lo[c] = of_ord(mn);
        if (hi) hi[c] = of_ord(mx);
    } else {
        const double sd = sqrt(s / (double)N);
        out0[c] = sd > 0.0 ? sd : 1.0;
    }
}

__global__ void k_zscore(double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ mean,
                         const double* __restrict__ sd) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d;
        const int c = (int)(e % d);
        X[r * ld + c] = (X[r * ld + c] - mean[c]) / sd[c];
    }
}

__device__ __forceinline__ int fine_of(double v, double lo, double hi) {
    if (!(hi > lo)) return 0;
    const double t = (v - lo) * (double)kFine / (hi - lo);
    int j = (int)floor(t);
    return j < 0 ? 0 : (j > kFine - 1 ? kFine - 1 : j);
}

__global__ void k_fine_hist(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ lo,
                            const double* __restrict__ hi, int* __restrict__ hist) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / d;
        const int c = (int)(e % d);
        atomicAdd(&hist[(size_t)c * kFine + fine_of(X[r * ld + c], lo[c], hi[c])], 1);
    }
}

// per column: quantile bin of every fine bin (one block per column)
__global__ void __launch_bounds__(1024) k_quantile_map(const int* __restrict__ hist, int64_t N, int B,
                                                       unsigned char* __restrict__ qmap) {
    __shared__ long long part[1024];
    const int c = blockIdx.x;
    const int* h = hist + (size_t)c * kFine;
    constexpr int per = kFine / 1024;
    long long local = 0;
    for (int k = 0; k < per; k++) local += h[threadIdx.x * per + k];
    part[threadIdx.x] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {      // inclusive scan of the thread totals
        const long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long C = part[threadIdx.x] - local;        // count below this thread's first fine bin
    for (int k = 0; k < per; k++) {
        const int j = threadIdx.x * per + k;
        const long long cj = h[j];
        long long q = ((long long)B * (2 * C + cj)) / (2 * N);
        if (q > B - 1) q = B - 1;
        qmap[(size_t)c * kFine + j] = (unsigned char)q;
        C += cj;
    }
}

// joint counts (quantile bin, class) per column; labels outside [0, nclass) are counted in bad
__global__ void __launch_bounds__(kThreads)
k_joint(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ lo,
        const double* __restrict__ hi, const unsigned char* __restrict__ qmap, const int32_t* __restrict__ labels,
        int B, int nclass, unsigned long long* __restrict__ joint, unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned int* sj = reinterpret_cast<unsigned int*>(sm);
    const int cells = d * B * nclass;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) sj[i] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kStatRows;
    const int64_t rows = (N - r0 < kStatRows) ? (N - r0) : kStatRows;
    for (int64_t e = threadIdx.x; e < rows * d; e += blockDim.x) {
        const int64_t r = r0 + e / d;
        const int c = (int)(e % d);
        const int y = labels[r];
        if (y < 0 || y >= nclass) {
            if (c == 0) atomicAdd(bad, 1ull);
            continue;
        }
        const int q = qmap[(size_t)c * kFine + fine_of(X[r * ld + c], lo[c], hi[c])];
        atomicAdd(&sj[(c * B + q) * nclass + y], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x)
        if (sj[i]) atomicAdd(&joint[i], (unsigned long long)sj[i]);
}

}  // namespace anova

using namespace anova;

namespace {

struct ColStats {
    double *mean = nullptr, *lo = nullptr, *hi = nullptr, *psum = nullptr;
    unsigned long long *pmin = nullptr, *pmax = nullptr;
    int nblk = 0;
};

anova_status col_stats(const double* X, int64_t N, int d, int64_t ld, ColStats& cs, cudaStream_t st) {
    cs.nblk = (int)((N + kStatRows - 1) / kStatRows);
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.psum, (size_t)cs.nblk * d * sizeof(double), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.pmin, (size_t)cs.nblk * d * sizeof(unsigned long long), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.pmax, (size_t)cs.nblk * d * sizeof(unsigned long long), st));
    const size_t sh = (size_t)d * 24;
    k_col_partials<<<cs.nblk, kThreads, sh, st>>>(X, N, d, ld, nullptr, 0, cs.psum, cs.pmin, cs.pmax);
    k_col_totals<<<(d + 255) / 256, 256, 0, st>>>(cs.psum, cs.pmin, cs.pmax, cs.nblk, d, N, 0, cs.mean, cs.lo, cs.hi);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

void col_stats_free(ColStats& cs, cudaStream_t st) {
    cudaFreeAsync(cs.psum, st);
    cudaFreeAsync(cs.pmin, st);
    cudaFreeAsync(cs.pmax, st);
}

bool shapes_ok(const double* X, int64_t N, int32_t d, int64_t ld) {
    return X && N >= 1 && d >= 1 && d <= kFeatMaxD && ld >= d;
}

}  // namespace

extern "C" {

anova_status anova_zscore_fit(const double* X, int64_t N, int32_t d, int64_t ld, double* mean, double* sd,
                              void* stream) {
    if (!shapes_ok(X, N, d, ld) || !mean || !sd) {
        set_error("anova_zscore_fit: need N >= 1, 1 <= d <= 2048, ld >= d and device pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ColStats cs;
    cs.mean = mean;
    anova_status s = col_stats(X, N, d, ld, cs, st);
    if (s == ANOVA_OK) {
        k_col_partials<<<cs.nblk, kThreads, (size_t)d * 24, st>>>(X, N, d, ld, mean, 1, cs.psum, nullptr, nullptr);
        k_col_totals<<<(d + 255) / 256, 256, 0, st>>>(cs.psum, nullptr, nullptr, cs.nblk, d, N, 1, sd, nullptr,
                                                      nullptr);
        if (cudaGetLastError() != cudaSuccess) s = ANOVA_ECUDA;
    }
    col_stats_free(cs, st);
    return s;
}

anova_status anova_zscore_apply(double* X, int64_t N, int32_t d, int64_t ld, const double* mean, const double* sd,
                                void* stream) {
    if (!shapes_ok(X, N, d, ld) || !mean || !sd) {
        set_error("anova_zscore_apply: need N >= 1, 1 <= d <= 2048, ld >= d and device pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_zscore<<<grid_for(N * d, kThreads, 16 * 152), kThreads, 0, st>>>(X, N, d, ld, mean, sd);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

anova_status anova_mis(const double* X, int64_t N, int32_t d, int64_t ld, const int32_t* labels, int32_t nclass,
                       int32_t bins, double* mis, void* stream) {
    if (!shapes_ok(X, N, d, ld) || !labels || !mis || nclass < 1 || nclass > kMaxClasses || bins < 1 ||
        bins > kMaxQBins || (size_t)d * bins * nclass * 4 > 200 * 1024) {
        set_error("anova_mis: need N >= 1, 1 <= d <= 2048, ld >= d, 1 <= nclass <= 64, 1 <= bins <= 64, "
                  "d * bins * nclass <= 51200 and valid pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ColStats cs;
    int* hist = nullptr;
    unsigned char* qmap = nullptr;
    unsigned long long *joint = nullptr, *bad = nullptr;
    const size_t cells = (size_t)d * bins * nclass;
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.mean, d * sizeof(double), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.lo, d * sizeof(double), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&cs.hi, d * sizeof(double), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&hist, (size_t)d * kFine * sizeof(int), st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&qmap, (size_t)d * kFine, st));
    ANOVA_CUDA_TRY(cudaMallocAsync(&joint, (cells + 1) * sizeof(unsigned long long), st));
    bad = joint + cells;
    anova_status s = col_stats(X, N, d, ld, cs, st);
    std::vector<unsigned long long> hj(cells + 1);
    if (s == ANOVA_OK) {
        cudaMemsetAsync(hist, 0, (size_t)d * kFine * sizeof(int), st);
        cudaMemsetAsync(joint, 0, (cells + 1) * sizeof(unsigned long long), st);
        k_fine_hist<<<grid_for(N * d, kThreads, 16 * 152), kThreads, 0, st>>>(X, N, d, ld, cs.lo, cs.hi, hist);
        k_quantile_map<<<d, 1024, 0, st>>>(hist, N, bins, qmap);
        static bool attr = [] {
            cudaFuncSetAttribute(k_joint, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            return true;
        }();
        (void)attr;
        k_joint<<<cs.nblk, kThreads, cells * sizeof(unsigned int), st>>>(X, N, d, ld, cs.lo, cs.hi, qmap, labels,
                                                                        bins, nclass, joint, bad);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hj.data(), joint, (cells + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("anova_mis: ") + cudaGetErrorString(e));
            s = ANOVA_ECUDA;
        }
    }
    col_stats_free(cs, st);
    cudaFreeAsync(cs.mean, st);
    cudaFreeAsync(cs.lo, st);
    cudaFreeAsync(cs.hi, st);
    cudaFreeAsync(hist, st);
    cudaFreeAsync(qmap, st);
    cudaFreeAsync(joint, st);
    if (s != ANOVA_OK) return s;
    if (hj[cells] != 0) {
        set_error("anova_mis: " + std::to_string(hj[cells]) + " labels outside [0, nclass)");
        return ANOVA_EINVAL;
    }
    // the score from the joint counts (host, FP64, fixed order)
    for (int c = 0; c < d; c++) {
        const unsigned long long* n = hj.data() + (size_t)c * bins * nclass;
        std::vector<double> nq(bins, 0.0), ny(nclass, 0.0);
        for (int q = 0; q < bins; q++)
            for (int y = 0; y < nclass; y++) {
                nq[q] += (double)n[q * nclass + y];
                ny[y] += (double)n[q * nclass + y];
            }
        double v = 0.0;
        for (int q = 0; q < bins; q++)
            for (int y = 0; y < nclass; y++) {
                const double nqy = (double)n[q * nclass + y];
                if (nqy > 0.0) v += (nqy / (double)N) * std::log((double)N * nqy / (nq[q] * ny[y]));
            }
        mis[c] = v;
    }
    return ANOVA_OK;
}

anova_status anova_windows_from_mis(const double* mis, int32_t d, double threshold, int32_t* windows, int32_t* P) {
    if (!mis || d < 1 || !windows || !P) {
        set_error("anova_windows_from_mis: bad arguments");
        return ANOVA_EINVAL;
    }
    for (int f = 0; f < d; f++)
        if (!std::isfinite(mis[f])) {   // the ranking needs a total order of the scores
            set_error("anova_windows_from_mis: score " + std::to_string(f) + " is not finite");
            return ANOVA_EINVAL;
        }
    std::vector<int> order(d);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mis[a] > mis[b]; });
    std::vector<int> keep;
    for (int f : order)
        if (mis[f] >= threshold) keep.push_back(f);
    int p = 0;
    for (size_t i = 0; i < keep.size(); i += 3, p++)
        for (int t = 0; t < 3; t++) windows[3 * p + t] = (i + t < keep.size()) ? keep[i + t] : -1;
    *P = p;
    return ANOVA_OK;
}

}  // extern "C"
