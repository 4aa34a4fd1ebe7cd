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

// Element (r, c) of a block's rows goes to a fixed thread: with d <= 256 the
// block reads G = 256 / d rows per step, thread t < G d owning column t mod d
// and rows r0 + t / d, r0 + t / d + G, ... (a warp reads consecutive elements);
// with d > 256 thread t owns columns t, t + 256, ... of every row.  Each thread
// accumulates its columns in registers; the G threads of a column are summed in
// a fixed order in shared memory.  Per block: column sums of x (mode 0, with
// min and max) or of (x - mean)^2 (mode 1).
constexpr int kColsPerThread = (kFeatMaxD + kThreads - 1) / kThreads;

__global__ void __launch_bounds__(kThreads)
k_col_partials(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ mean, int mode,
               int64_t rows_per_block, double* __restrict__ psum, unsigned long long* __restrict__ pmin,
               unsigned long long* __restrict__ pmax) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int t = threadIdx.x;
    const int G = d <= kThreads ? kThreads / d : 1;          // rows per step
    const int active = d <= kThreads ? G * d : kThreads;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    double sum[kColsPerThread];
    unsigned long long mn[kColsPerThread], mx[kColsPerThread];
#pragma unroll
    for (int k = 0; k < kColsPerThread; k++) {
        sum[k] = 0.0;
        mn[k] = ~0ull;
        mx[k] = 0ull;
    }
    if (t < active) {
        const int g = d <= kThreads ? t / d : 0;
        const int c0 = d <= kThreads ? t % d : t;
        for (int64_t r = r0 + g; r < r1; r += G) {
            const double* row = X + r * ld;
#pragma unroll
            for (int k = 0; k < kColsPerThread; k++) {
                const int c = c0 + k * kThreads;
                if (k > 0 && (d <= kThreads || c >= d)) break;
                const double v = row[c];
                if (mode == 0) {
                    sum[k] += v;
                    const unsigned long long o = ord_of(v);
                    mn[k] = o < mn[k] ? o : mn[k];
                    mx[k] = o > mx[k] ? o : mx[k];
                } else {
                    const double dv = v - mean[c];
                    sum[k] = fma(dv, dv, sum[k]);
                }
            }
        }
    }
    if (d <= kThreads) {
        // fixed-order sum over the G threads of each column
        double* ssum = reinterpret_cast<double*>(sm);
        unsigned long long* smin = reinterpret_cast<unsigned long long*>(ssum + active);
        unsigned long long* smax = smin + active;
        if (t < active) {
            ssum[t] = sum[0];
            smin[t] = mn[0];
            smax[t] = mx[0];
        }
        __syncthreads();
        for (int c = t; c < d; c += kThreads) {
            double sc = 0.0;
            unsigned long long a = ~0ull, z = 0ull;
            for (int g = 0; g < G; g++) {
                sc += ssum[g * d + c];
                a = smin[g * d + c] < a ? smin[g * d + c] : a;
                z = smax[g * d + c] > z ? smax[g * d + c] : z;
            }
            psum[(size_t)blockIdx.x * d + c] = sc;
            if (mode == 0) {
                pmin[(size_t)blockIdx.x * d + c] = a;
                pmax[(size_t)blockIdx.x * d + c] = z;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kColsPerThread; k++) {
            const int c = t + k * kThreads;
            if (c >= d) break;
            psum[(size_t)blockIdx.x * d + c] = sum[k];
            if (mode == 0) {
                pmin[(size_t)blockIdx.x * d + c] = mn[k];
                pmax[(size_t)blockIdx.x * d + c] = mx[k];
            }
        }
    }
}

// column totals over the blocks, one block per column: thread t sums the
// partials of blocks t, t + 256, ... in order, then a fixed tree over the
// threads (deterministic); mode 0: mean, lo, hi; mode 1: std
__global__ void __launch_bounds__(kThreads)
k_col_totals(const double* __restrict__ psum, const unsigned long long* __restrict__ pmin,
             const unsigned long long* __restrict__ pmax, int nblk, int d, int64_t N, int mode,
             double* __restrict__ out0, double* __restrict__ lo, double* __restrict__ hi) {
    __shared__ double ss[kThreads];
    __shared__ unsigned long long smn[kThreads], smx[kThreads];
    const int c = blockIdx.x, t = threadIdx.x;
    double s = 0.0;
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int b = t; b < nblk; b += kThreads) {
        s += psum[(size_t)b * d + c];
        if (mode == 0) {
            const unsigned long long a = pmin[(size_t)b * d + c], z = pmax[(size_t)b * d + c];
            mn = a < mn ? a : mn;
            mx = z > mx ? z : mx;
        }
    }
    ss[t] = s;
    smn[t] = mn;
    smx[t] = mx;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            ss[t] += ss[t + h];
            smn[t] = smn[t + h] < smn[t] ? smn[t + h] : smn[t];
            smx[t] = smx[t + h] > smx[t] ? smx[t + h] : smx[t];
        }
        __syncthreads();
    }
    if (t != 0) return;
    if (mode == 0) {
        out0[c] = ss[0] / (double)N;
        if (lo) lo[c] = of_ord(smn[0]);
        if (hi) hi[c] = of_ord(smx[0]);
    } else {
        const double sd = sqrt(ss[0] / (double)N);
        out0[c] = sd > 0.0 ? sd : 1.0;
    }
}

// x = (x - mean) / sd in place, elements owned as in k_col_partials
__global__ void __launch_bounds__(kThreads)
k_zscore(double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ mean,
         const double* __restrict__ sd, int64_t rows_per_block) {
    const int t = threadIdx.x;
    const int G = d <= kThreads ? kThreads / d : 1;
    const int active = d <= kThreads ? G * d : kThreads;
    if (t >= active) return;
    const int g = d <= kThreads ? t / d : 0;
    const int c0 = d <= kThreads ? t % d : t;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    double m[kColsPerThread], s[kColsPerThread];
#pragma unroll
    for (int k = 0; k < kColsPerThread; k++) {
        const int c = c0 + k * kThreads;
        const bool ok = k == 0 || (d > kThreads && c < d);
        m[k] = ok ? mean[c] : 0.0;
        s[k] = ok ? sd[c] : 1.0;
    }
    for (int64_t r = r0 + g; r < r1; r += G) {
        double* row = X + r * ld;
#pragma unroll
        for (int k = 0; k < kColsPerThread; k++) {
            const int c = c0 + k * kThreads;
            if (k > 0 && (d <= kThreads || c >= d)) break;
            row[c] = (row[c] - m[k]) / s[k];
        }
    }
}

__device__ __forceinline__ int fine_of(double v, double lo, double hi) {
    if (!(hi > lo)) return 0;
    const double t = (v - lo) * (double)kFine / (hi - lo);
    int j = (int)floor(t);
    return j < 0 ? 0 : (j > kFine - 1 ? kFine - 1 : j);
}

// MIS histograms: warp w of a block takes columns w, w + 8, ... of the block's
// rows in groups of 32 (lane = row), so the values a warp holds belong to one
// column and equal histogram cells are combined (__match_any_sync) before the
// one atomic add per distinct cell.
constexpr int kHistWarps = kThreads / 32;

__device__ __forceinline__ void add_aggregated(unsigned int* base, int key, bool valid) {
    const unsigned int act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned int same = __match_any_sync(act, key);
    if ((__ffs(same) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&base[key], (unsigned int)__popc(same));
}

__global__ void __launch_bounds__(kThreads)
k_fine_hist(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ lo,
            const double* __restrict__ hi, int64_t rows_per_block, unsigned int* __restrict__ hist) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    for (int64_t rb = r0; rb < r1; rb += 32) {
        const int64_t r = rb + lane;
        const bool in = r < r1;
        for (int c = warp; c < d; c += kHistWarps) {
            const double v = in ? X[r * ld + c] : 0.0;
            add_aggregated(hist, c * kFine + fine_of(v, lo[c], hi[c]), in);
        }
    }
}

// per column: quantile bin of every fine bin (one block per column)
__global__ void __launch_bounds__(1024) k_quantile_map(const unsigned int* __restrict__ hist, int64_t N, int B,
                                                       unsigned char* __restrict__ qmap) {
    __shared__ long long part[1024];
    const int c = blockIdx.x;
    const unsigned int* h = hist + (size_t)c * kFine;
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

// joint counts (quantile bin, class) per column in shared memory per block;
// labels outside [0, nclass) are counted in bad (once per row)
__global__ void __launch_bounds__(kThreads)
k_joint(const double* __restrict__ X, int64_t N, int d, int64_t ld, const double* __restrict__ lo,
        const double* __restrict__ hi, const unsigned char* __restrict__ qmap, const int32_t* __restrict__ labels,
        int B, int nclass, int64_t rows_per_block, unsigned long long* __restrict__ joint,
        unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned int* sj = reinterpret_cast<unsigned int*>(sm);
    const int cells = d * B * nclass;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) sj[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    unsigned int nbad = 0;
    for (int64_t rb = r0; rb < r1; rb += 32) {
        const int64_t r = rb + lane;
        const bool in = r < r1;
        const int y = in ? labels[r] : 0;
        const bool ok = in && y >= 0 && y < nclass;
        if (warp == 0 && in && !ok) nbad++;
        for (int c = warp; c < d; c += kHistWarps) {
            const double v = ok ? X[r * ld + c] : 0.0;
            const int q = ok ? qmap[(size_t)c * kFine + fine_of(v, lo[c], hi[c])] : 0;
            add_aggregated(sj, (c * B + q) * nclass + y, ok);
        }
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x)
        if (sj[i]) atomicAdd(&joint[i], (unsigned long long)sj[i]);
}

// blocks and rows per block of the statistics and histogram kernels: every block
// at least 256 rows, at most 8 blocks per SM
static void stat_grid(int64_t N, int sms, int* nblk, int64_t* rows) {
    int64_t b = std::min<int64_t>((N + 255) / 256, 8 * (int64_t)std::max(sms, 1));
    b = std::max<int64_t>(b, 1);
    *rows = ((N + b - 1) / b + 31) / 32 * 32;
    *nblk = (int)((N + *rows - 1) / *rows);
}

static int device_sms() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace anova

using namespace anova;

namespace {

// column statistics of one call: block partials (sums, min, max) and the grid
struct ColStats {
    double *psum = nullptr;
    unsigned long long *pmin = nullptr, *pmax = nullptr;
    int nblk = 0;
    int64_t rows = 0;
};

size_t partial_smem(int d) { return d <= kThreads ? (size_t)(kThreads / d) * d * 24 : 0; }

anova_status col_alloc(int64_t N, int d, ColStats& cs, Scratch& scratch) {
    stat_grid(N, device_sms(), &cs.nblk, &cs.rows);
    ANOVA_CUDA_TRY(scratch.alloc(&cs.psum, (size_t)cs.nblk * d * sizeof(double)));
    ANOVA_CUDA_TRY(scratch.alloc(&cs.pmin, (size_t)cs.nblk * d * sizeof(unsigned long long)));
    ANOVA_CUDA_TRY(scratch.alloc(&cs.pmax, (size_t)cs.nblk * d * sizeof(unsigned long long)));
    return ANOVA_OK;
}

// mean (and lo, hi when given) of every column: one read of X
anova_status col_mean(const double* X, int64_t N, int d, int64_t ld, const ColStats& cs, double* mean, double* lo,
                      double* hi, cudaStream_t st) {
    k_col_partials<<<cs.nblk, kThreads, partial_smem(d), st>>>(X, N, d, ld, nullptr, 0, cs.rows, cs.psum, cs.pmin,
                                                               cs.pmax);
    k_col_totals<<<d, kThreads, 0, st>>>(cs.psum, cs.pmin, cs.pmax, cs.nblk, d, N, 0, mean, lo, hi);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
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
    Scratch scratch(st);
    ColStats cs;
    ANOVA_TRY(col_alloc(N, d, cs, scratch));
    ANOVA_TRY(col_mean(X, N, d, ld, cs, mean, nullptr, nullptr, st));
    // second pass: sums of squared deviations from the mean (the two-pass form)
    k_col_partials<<<cs.nblk, kThreads, partial_smem(d), st>>>(X, N, d, ld, mean, 1, cs.rows, cs.psum, nullptr,
                                                               nullptr);
    k_col_totals<<<d, kThreads, 0, st>>>(cs.psum, nullptr, nullptr, cs.nblk, d, N, 1, sd, nullptr, nullptr);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

anova_status anova_zscore_apply(double* X, int64_t N, int32_t d, int64_t ld, const double* mean, const double* sd,
                                void* stream) {
    if (!shapes_ok(X, N, d, ld) || !mean || !sd) {
        set_error("anova_zscore_apply: need N >= 1, 1 <= d <= 2048, ld >= d and device pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int nblk = 0;
    int64_t rows = 0;
    stat_grid(N, device_sms(), &nblk, &rows);
    k_zscore<<<nblk, kThreads, 0, st>>>(X, N, d, ld, mean, sd, rows);
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
    Scratch scratch(st);
    ColStats cs;
    double *mean = nullptr, *lo = nullptr, *hi = nullptr;
    unsigned int* hist = nullptr;
    unsigned char* qmap = nullptr;
    unsigned long long *joint = nullptr, *bad = nullptr;
    const size_t cells = (size_t)d * bins * nclass;
    ANOVA_TRY(col_alloc(N, d, cs, scratch));
    ANOVA_CUDA_TRY(scratch.alloc(&mean, d * sizeof(double)));
    ANOVA_CUDA_TRY(scratch.alloc(&lo, d * sizeof(double)));
    ANOVA_CUDA_TRY(scratch.alloc(&hi, d * sizeof(double)));
    ANOVA_CUDA_TRY(scratch.alloc(&hist, (size_t)d * kFine * sizeof(unsigned int)));
    ANOVA_CUDA_TRY(scratch.alloc(&qmap, (size_t)d * kFine));
    ANOVA_CUDA_TRY(scratch.alloc(&joint, (cells + 1) * sizeof(unsigned long long)));
    bad = joint + cells;
    ANOVA_TRY(col_mean(X, N, d, ld, cs, mean, lo, hi, st));
    std::vector<unsigned long long> hj(cells + 1);
    ANOVA_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)d * kFine * sizeof(unsigned int), st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(joint, 0, (cells + 1) * sizeof(unsigned long long), st));
    k_fine_hist<<<cs.nblk, kThreads, 0, st>>>(X, N, d, ld, lo, hi, cs.rows, hist);
    k_quantile_map<<<d, 1024, 0, st>>>(hist, N, bins, qmap);
    static bool attr = [] {
        cudaFuncSetAttribute(k_joint, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)attr;
    k_joint<<<cs.nblk, kThreads, cells * sizeof(unsigned int), st>>>(X, N, d, ld, lo, hi, qmap, labels, bins, nclass,
                                                                    cs.rows, joint, bad);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemcpyAsync(hj.data(), joint, (cells + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                   st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
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
