// features.cu -- window construction upstream of the fast summation
// (arXiv 2111.10140, Sec. 5: features ranked by mutual information score,
// those below a threshold dropped, the rest grouped three at a time in rank
// order; Sec. 6.1: z-score normalisation with training statistics).
//
// Column statistics read the row-major matrix in coalesced row blocks with
// per-thread column accumulators; the blocks' partials are combined in a
// fixed order (deterministic).  The z-score fit is one read of X: per block
// and column the sums of x - K and (x - K)^2 with a shift K taken from the
// block's first row, combined over blocks by the pairwise mean / M2 update.
// The score is the plug-in mutual information between the label and the
// feature's quantile bin, the quantile bins coming from a fine equal-width
// histogram (bin of a value: floor((v - lo) F / (hi - lo)), F = 4096, the last
// bin closed; quantile bin of fine bin j: floor(B (2 C_j + c_j) / (2 N)) with
// C_j the count below j and c_j its own count, in integers).  The fine bin is
// a non-decreasing function of v, so it is computed exactly from per-column
// thresholds (found once per column in FP64 from the definition) by integer
// comparisons of order keys: no FP64 division per element, the same bins as
// the definition evaluated in FP64.
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
// and rows r0 + t / d, r0 + t / d + G, ... (a warp reads consecutive elements;
// four rows' loads in flight per step); with d > 256 thread t owns columns t,
// t + 256, ... of every row.  Each thread accumulates its columns in
// registers; the G threads of a column are combined in a fixed order in
// shared memory.
constexpr int kColsPerThread = (kFeatMaxD + kThreads - 1) / kThreads;

// Per block and column, one read of X:
//   kMoments  S = sum (x - K), Q = sum (x - K)^2 with the shift K = the
//             column's value in the block's first row (same K for every thread
//             of the block, so the thread sums add directly);
//   kRange    min and max as order-preserving integer keys (no FP64 work).
enum ColMode { kMoments = 0, kRange = 1 };

template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_col_partials(const double* __restrict__ X, int64_t N, int d, int64_t ld, int64_t rows_per_block,
               double* __restrict__ pS, double* __restrict__ pQ, double* __restrict__ pK,
               unsigned long long* __restrict__ pmin, unsigned long long* __restrict__ pmax) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int t = threadIdx.x;
    const int G = d <= kThreads ? kThreads / d : 1;          // rows per step
    const int active = d <= kThreads ? G * d : kThreads;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    double S[kColsPerThread], Q[kColsPerThread], K[kColsPerThread];
    unsigned long long mn[kColsPerThread], mx[kColsPerThread];
    const int g = d <= kThreads ? t / d : 0;
    const int c0 = d <= kThreads ? t % d : t;
#pragma unroll
    for (int k = 0; k < kColsPerThread; k++) {
        S[k] = 0.0;
        Q[k] = 0.0;
        K[k] = 0.0;
        mn[k] = ~0ull;
        mx[k] = 0ull;
    }
    if (t < active) {
        if (MODE == kMoments) {
#pragma unroll
            for (int k = 0; k < kColsPerThread; k++) {
                const int c = c0 + k * kThreads;
                if (k > 0 && (d <= kThreads || c >= d)) break;
                K[k] = X[r0 * ld + c];
            }
        }
        auto take = [&](double v, int k) {
            if (MODE == kMoments) {
                const double dv = v - K[k];
                S[k] += dv;
                Q[k] = fma(dv, dv, Q[k]);
            } else {
                const unsigned long long o = ord_of(v);
                mn[k] = o < mn[k] ? o : mn[k];
                mx[k] = o > mx[k] ? o : mx[k];
            }
        };
        if (d <= kThreads) {
            const double* col = X + c0;
            int64_t r = r0 + g;
            for (; r + 3 * G < r1; r += 4 * G) {
                const double v0 = col[r * ld], v1 = col[(r + G) * ld], v2 = col[(r + 2 * G) * ld],
                             v3 = col[(r + 3 * G) * ld];
                take(v0, 0);
                take(v1, 0);
                take(v2, 0);
                take(v3, 0);
            }
            for (; r < r1; r += G) take(col[r * ld], 0);
        } else {
            for (int64_t r = r0; r < r1; r++) {
                const double* row = X + r * ld;
#pragma unroll
                for (int k = 0; k < kColsPerThread; k++) {
                    const int c = c0 + k * kThreads;
                    if (c >= d) break;
                    take(row[c], k);
                }
            }
        }
    }
    const size_t o = (size_t)blockIdx.x * d;
    if (d <= kThreads) {
        // fixed-order combination of the G threads of each column
        double* s0 = reinterpret_cast<double*>(sm);
        double* s1 = s0 + active;
        unsigned long long* u0 = reinterpret_cast<unsigned long long*>(sm);
        unsigned long long* u1 = u0 + active;
        if (t < active) {
            if (MODE == kMoments) {
                s0[t] = S[0];
                s1[t] = Q[0];
            } else {
                u0[t] = mn[0];
                u1[t] = mx[0];
            }
        }
        __syncthreads();
        for (int c = t; c < d; c += kThreads) {
            if (MODE == kMoments) {
                double a = 0.0, b = 0.0;
                for (int h = 0; h < G; h++) {
                    a += s0[h * d + c];
                    b += s1[h * d + c];
                }
                pS[o + c] = a;
                pQ[o + c] = b;
                pK[o + c] = X[r0 * ld + c];
            } else {
                unsigned long long a = ~0ull, z = 0ull;
                for (int h = 0; h < G; h++) {
                    a = u0[h * d + c] < a ? u0[h * d + c] : a;
                    z = u1[h * d + c] > z ? u1[h * d + c] : z;
                }
                pmin[o + c] = a;
                pmax[o + c] = z;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kColsPerThread; k++) {
            const int c = t + k * kThreads;
            if (c >= d) break;
            if (MODE == kMoments) {
                pS[o + c] = S[k];
                pQ[o + c] = Q[k];
                pK[o + c] = K[k];
            } else {
                pmin[o + c] = mn[k];
                pmax[o + c] = mx[k];
            }
        }
    }
}

// (count, mean, sum of squared deviations) of two disjoint row sets combined
// (the pairwise update of Chan, Golub and LeVeque)
struct Moments {
    double n, mean, m2;
};
__device__ __forceinline__ Moments merge(const Moments& a, const Moments& b) {
    if (a.n == 0.0) return b;
    if (b.n == 0.0) return a;
    const double n = a.n + b.n;
    const double delta = b.mean - a.mean;
    return {n, a.mean + delta * (b.n / n), a.m2 + b.m2 + delta * delta * (a.n * (b.n / n))};
}

// column totals, one block per column: thread t combines the partials of
// blocks t, t + 256, ... in order, then a fixed tree over the threads
// (deterministic).  kMoments: mean and sd (divisor N, sd = 1 for a constant
// column); kRange: lo and hi.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_col_totals(const double* __restrict__ pS, const double* __restrict__ pQ, const double* __restrict__ pK,
             const unsigned long long* __restrict__ pmin, const unsigned long long* __restrict__ pmax, int nblk,
             int d, int64_t N, int64_t rows_per_block, double* __restrict__ out0, double* __restrict__ out1) {
    __shared__ Moments sm_m[kThreads];
    __shared__ unsigned long long smn[kThreads], smx[kThreads];
    const int c = blockIdx.x, t = threadIdx.x;
    Moments acc = {0.0, 0.0, 0.0};
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int b = t; b < nblk; b += kThreads) {
        const size_t i = (size_t)b * d + c;
        if (MODE == kMoments) {
            const int64_t r0 = (int64_t)b * rows_per_block;
            const double nb = (double)(min(N, r0 + rows_per_block) - r0);
            const double S = pS[i];
            const double m2 = pQ[i] - S * (S / nb);
            acc = merge(acc, Moments{nb, pK[i] + S / nb, m2 > 0.0 ? m2 : 0.0});
        } else {
            mn = pmin[i] < mn ? pmin[i] : mn;
            mx = pmax[i] > mx ? pmax[i] : mx;
        }
    }
    sm_m[t] = acc;
    smn[t] = mn;
    smx[t] = mx;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            if (MODE == kMoments) {
                sm_m[t] = merge(sm_m[t], sm_m[t + h]);
            } else {
                smn[t] = smn[t + h] < smn[t] ? smn[t + h] : smn[t];
                smx[t] = smx[t + h] > smx[t] ? smx[t + h] : smx[t];
            }
        }
        __syncthreads();
    }
    if (t != 0) return;
    if (MODE == kMoments) {
        out0[c] = sm_m[0].mean;
        const double sd = sqrt(sm_m[0].m2 / (double)N);
        out1[c] = sd > 0.0 ? sd : 1.0;
    } else {
        out0[c] = of_ord(smn[0]);
        out1[c] = of_ord(smx[0]);
    }
}

// x = (x - mean) * (1 / sd) in place (two FP64 operations per element; within
// 1.5 units in the last place of the quotient), elements owned as in
// k_col_partials
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
        s[k] = ok ? 1.0 / sd[c] : 1.0;
    }
    if (d <= kThreads) {
        double* col = X + c0;
        int64_t r = r0 + g;
        for (; r + 3 * G < r1; r += 4 * G) {
            const double v0 = col[r * ld], v1 = col[(r + G) * ld], v2 = col[(r + 2 * G) * ld],
                         v3 = col[(r + 3 * G) * ld];
            col[r * ld] = (v0 - m[0]) * s[0];
            col[(r + G) * ld] = (v1 - m[0]) * s[0];
            col[(r + 2 * G) * ld] = (v2 - m[0]) * s[0];
            col[(r + 3 * G) * ld] = (v3 - m[0]) * s[0];
        }
        for (; r < r1; r += G) col[r * ld] = (col[r * ld] - m[0]) * s[0];
        return;
    }
    for (int64_t r = r0; r < r1; r++) {
        double* row = X + r * ld;
#pragma unroll
        for (int k = 0; k < kColsPerThread; k++) {
            const int c = c0 + k * kThreads;
            if (c >= d) break;
            row[c] = (row[c] - m[k]) * s[k];
        }
    }
}

// The fine bin is a non-decreasing function of v, so it is fixed by the
// thresholds thr_j = the smallest double v (as an order key) with bin >= j:
// bin(v) = max{ j : thr_j <= key(v) }.  Row c of the table holds thr_0 = 0 (no
// key below), thr_1 .. thr_{F-1}, and thr_F = ~0 (no key reaches it).  The bin
// depends on v only through the rounded difference D = RN(v - lo), so each
// threshold takes two monotone searches: the smallest difference D* in
// [0, hi - lo] whose bin RN(D F / (hi - lo)) reaches j (the guess j (hi - lo) /
// F is within a few units in the last place of it), then the smallest v in
// [lo, hi] with RN(v - lo) >= D* (one subtraction per probe).  Both start from
// a guess and gallop, then bisect, over the order keys.
constexpr int kThrRow = kFine + 1;

// smallest key in [klo, khi] where pred holds (pred monotone, pred(khi) true),
// searched from the guess k0
template <typename Pred>
__device__ unsigned long long smallest_key(unsigned long long klo, unsigned long long khi, unsigned long long k0,
                                           Pred pred) {
    k0 = k0 < klo ? klo : (k0 > khi ? khi : k0);
    unsigned long long a, b;   // !pred(a) (or a == klo untested), pred(b), a < b
    if (pred(k0)) {
        b = k0;
        unsigned long long step = 1;
        for (;;) {
            if (b - klo < step) {
                if (pred(klo)) return klo;
                a = klo;
                break;
            }
            const unsigned long long q = b - step;
            if (pred(q)) {
                b = q;
                step <<= 1;
            } else {
                a = q;
                break;
            }
        }
    } else {
        a = k0;
        unsigned long long step = 1;
        for (;;) {
            if (khi - a <= step) {
                b = khi;
                break;
            }
            const unsigned long long q = a + step;
            if (pred(q)) {
                b = q;
                break;
            }
            a = q;
            step <<= 1;
        }
    }
    while (b - a > 1) {
        const unsigned long long q = a + (b - a) / 2;
        if (pred(q)) b = q;
        else a = q;
    }
    return b;
}

__device__ unsigned long long threshold_key(int j, double lo, double hi) {
    const double h = hi - lo;
    // bin of a rounded difference D, as the definition evaluates it
    auto bin_of_d = [&](double D) {
        int b = (int)floor(D * (double)kFine / h);
        return b < 0 ? 0 : (b > kFine - 1 ? kFine - 1 : b);
    };
    const unsigned long long dstar = smallest_key(ord_of(0.0), ord_of(h), ord_of((double)j * (h / (double)kFine)),
                                                  [&](unsigned long long k) { return bin_of_d(of_ord(k)) >= j; });
    const double D = of_ord(dstar);
    return smallest_key(ord_of(lo), ord_of(hi), ord_of(lo + D),
                        [&](unsigned long long k) { return of_ord(k) - lo >= D; });
}

// thresholds of every column (one thread per (column, j)) and the column's
// FP32 screen: x = lo, y = F / (hi - lo) (the estimate t = (v - lo) y in FP32),
// z = delta, a bound on |t - t_def| where t_def is the definition's FP64
// quotient.  With M = max(|lo|, |hi|): the 20-bit truncation of v and the
// rounding of lo to FP32 move t by at most (F / h) M (2^-20 + 2^-24); the FP32
// subtraction, the rounding of F / h and the product by at most 3.1 2^-24 F
// (< 8e-4); denormal v (read as 0) by (F / h) 2^-126; the definition's own
// FP64 roundings by < 1e-12.  delta = 1.25 (first and third) + 1e-3.  Where
// the FP32 form cannot hold the column (|values| or F / h beyond 1e37) or
// delta >= 1/4, z = 1: every element goes to the thresholds.
__global__ void __launch_bounds__(kThreads)
k_fine_thresholds(const double* __restrict__ lo, const double* __restrict__ hi, int d,
                  unsigned long long* __restrict__ thr, float4* __restrict__ screen) {
    const int c = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d || j > kFine) return;
    const double L = lo[c], H = hi[c];
    unsigned long long key;
    if (j == 0) key = 0ull;
    else if (j == kFine || !(H > L)) key = ~0ull;
    else key = threshold_key(j, L, H);
    thr[(size_t)c * kThrRow + j] = key;
    if (j == 0) {
        if (H > L) {
            const double M = fmax(fabs(L), fabs(H)), sfd = (double)kFine / (H - L);
            double delta = 1.25 * (sfd * M * (0x1p-20 + 0x1p-24) + sfd * 0x1p-126) + 1e-3;
            if (!(M < 1e37) || !(sfd < 1e37) || !(delta < 0.25)) delta = 1.0;
            screen[c] = make_float4((float)L, (float)sfd, __double2float_ru(delta), 0.f);
        } else {
            screen[c] = make_float4(0.f, 0.f, 0.f, 0.f);   // constant column: t = 0, bin 0 for every value
        }
    }
}

// FP32 value of v from its high word (mantissa truncated to 20 bits), 0 where
// the exponent is outside FP32's normal range: only a starting point
__device__ __forceinline__ float approx_float(double v) {
    const int h = __double2hiint(v);
    const int e = (h >> 20) & 0x7ff;
    if (e <= 896 || e >= 1151) return 0.0f;
    return __int_as_float((h & (int)0x80000000) | (((h & 0x7fffffff) - (896 << 20)) << 3));
}

// fine bin of v from the thresholds of its column: an FP32 estimate, then
// moved until thr_j <= key(v) < thr_{j+1} (exact; each loop ends within F steps)
__device__ __forceinline__ int screen_bin(double v, float4 scr) {
    const float t = (approx_float(v) - scr.x) * scr.y;
    return (int)fminf(fmaxf(t, 0.0f), (float)(kFine - 1));
}
// the bin from the FP32 estimate alone where it is at least delta from every
// bin boundary (then the definition's bin is the same), else -1
__device__ __forceinline__ int fast_bin(double v, float4 scr) {
    const float t = (approx_float(v) - scr.x) * scr.y;
    const float dl = scr.z;
    if (!(dl < 0.5f) || !(t == t)) return -1;
    if (t < __fsub_rd(1.0f, dl)) return 0;                        // t_def < 1: bin 0 (clamped below)
    if (t >= __fadd_ru((float)(kFine - 1), dl)) return kFine - 1;  // t_def >= F - 1: the last bin
    const float fl = floorf(t);
    return (t - fl < dl || fl + 1.0f - t < dl) ? -1 : (int)fl;
}
__device__ __forceinline__ int fix_bin(unsigned long long key, int j, const unsigned long long* __restrict__ thr) {
    while (j > 0 && key < __ldg(thr + j)) j--;
    while (j < kFine - 1 && key >= __ldg(thr + j + 1)) j++;
    return j;
}
__device__ __forceinline__ int fine_bin(double v, const unsigned long long* __restrict__ thr, float4 scr) {
    const int j = fast_bin(v, scr);
    return j >= 0 ? j : fix_bin(ord_of(v), screen_bin(v, scr), thr);
}

// fine bin of every element (anova_mis_fine_bins), elements owned as in
// k_col_partials
__global__ void __launch_bounds__(kThreads)
k_fine_bins_out(const double* __restrict__ X, int64_t N, int d, int64_t ld,
                const unsigned long long* __restrict__ thr, const float4* __restrict__ screen,
                int64_t rows_per_block, int32_t* __restrict__ out) {
    const int t = threadIdx.x;
    const int G = d <= kThreads ? kThreads / d : 1;
    const int active = d <= kThreads ? G * d : kThreads;
    if (t >= active) return;
    const int g = d <= kThreads ? t / d : 0;
    const int c0 = d <= kThreads ? t % d : t;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    for (int64_t r = r0 + g; r < r1; r += G)
        for (int c = c0; c < d; c += (d <= kThreads ? d : kThreads))
            out[r * d + c] = fine_bin(X[r * ld + c], thr + (size_t)c * kThrRow, screen[c]);
}

// Three-pass MIS (any nclass): the fine histogram by global atomics, the
// quantile map, then the joint counts in shared memory per block.  Warp w of a
// block takes columns w, w + 8, ... of the block's rows in groups of 32 (lane
// = row), so the values a warp holds belong to one column and equal histogram
// cells are combined (__match_any_sync) before the one atomic add per
// distinct cell.
constexpr int kHistWarps = kThreads / 32;

__device__ __forceinline__ void add_aggregated(unsigned int* base, int key, bool valid) {
    const unsigned int act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned int same = __match_any_sync(act, key);
    if ((__ffs(same) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&base[key], (unsigned int)__popc(same));
}

__global__ void __launch_bounds__(kThreads)
k_fine_hist(const double* __restrict__ X, int64_t N, int d, int64_t ld, const unsigned long long* __restrict__ thr,
            const float4* __restrict__ screen, int64_t rows_per_block, unsigned int* __restrict__ hist) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    for (int64_t rb = r0; rb < r1; rb += 32) {
        const int64_t r = rb + lane;
        const bool in = r < r1;
        for (int c = warp; c < d; c += kHistWarps) {
            const double v = in ? X[r * ld + c] : 0.0;
            const int j = in ? fine_bin(v, thr + (size_t)c * kThrRow, screen[c]) : 0;
            add_aggregated(hist, c * kFine + j, in);
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
k_joint(const double* __restrict__ X, int64_t N, int d, int64_t ld, const unsigned long long* __restrict__ thr,
        const float4* __restrict__ screen, const unsigned char* __restrict__ qmap,
        const int32_t* __restrict__ labels, int B, int nclass, int64_t rows_per_block,
        unsigned long long* __restrict__ joint, unsigned long long* __restrict__ bad) {
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
            const int q = ok ? qmap[(size_t)c * kFine + fine_bin(v, thr + (size_t)c * kThrRow, screen[c])] : 0;
            add_aggregated(sj, (c * B + q) * nclass + y, ok);
        }
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x)
        if (sj[i]) atomicAdd(&joint[i], (unsigned long long)sj[i]);
}

// Two-pass MIS (nclass <= 4): one read of X gives the (fine bin, class)
// counts of every column, from which the quantile map and the joint
// (quantile bin, class) counts follow without reading X again.  Block (g, rr)
// takes column group g (gcols consecutive columns) over row range rr and
// counts in shared memory: per (column, fine bin) ceil(nclass / 2) 32-bit
// words holding two 16-bit class counts each (a block takes at most 65535
// rows, so a half never carries into the other), and one spare word after
// each column's counts, so that equal bins of neighbouring columns sit in
// different banks.  Thread t handles column
// t mod gc of rows t / gc, t / gc + NT / gc, ... (consecutive threads read
// consecutive columns of a row).  The block writes its counts to its own slot
// of a scratch array; k_class_hist_reduce adds the slots in a fixed order.
constexpr int kCHThreads = 512;
constexpr int kCHMaxRows = 65535;
constexpr size_t kCHSmem = 100 * 1024;                 // shared counts per block: two blocks per SM
constexpr size_t kCHPartMax = (size_t)512 << 20;       // largest scratch of block counts

__global__ void __launch_bounds__(kCHThreads)
k_fine_class_hist(const double* __restrict__ X, int64_t N, int d, int64_t ld,
                  const unsigned long long* __restrict__ thr, const float4* __restrict__ screen,
                  const int32_t* __restrict__ labels, int nclass, int gcols, int ngroups, int64_t rows_per_block,
                  unsigned int* __restrict__ part, unsigned long long* __restrict__ bad) {
    extern __shared__ __align__(16) unsigned int sh[];
    const int W = (nclass + 1) / 2;                       // words per (column, fine bin)
    const int CS = kFine * W + 1;                          // words per column: odd, so columns fall on other banks
    const int g = blockIdx.x % ngroups;
    const int64_t rr = blockIdx.x / ngroups;
    const int c_lo = g * gcols;
    const int gc = min(gcols, d - c_lo);
    const int words = gc * CS;
    for (int i = threadIdx.x; i < words; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const int64_t r0 = rr * rows_per_block;
    const int64_t r1 = min(N, r0 + rows_per_block);
    const int per = kCHThreads / gc;                      // rows per step
    const int cl = threadIdx.x % gc;
    const int c = c_lo + cl;
    unsigned int nbad = 0;
    if (threadIdx.x < per * gc) {
        const unsigned long long* __restrict__ tc = thr + (size_t)c * kThrRow;
        const float4 scr = screen[c];
        // four rows per step, their loads in flight together; an element near a bin
        // boundary (rare) takes its bin from the thresholds
        constexpr int U = 4;
        for (int64_t r = r0 + threadIdx.x / gc; r < r1; r += U * per) {
            double v[U];
            int y[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t ru = r + (int64_t)u * per;
                const bool in = ru < r1;
                y[u] = in ? labels[ru] : -1;
                v[u] = in ? X[ru * ld + c] : 0.0;
                if (in && (y[u] < 0 || y[u] >= nclass) && g == 0 && cl == 0) nbad++;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (y[u] < 0 || y[u] >= nclass) continue;
                int j = fast_bin(v[u], scr);
                if (j < 0) j = fix_bin(ord_of(v[u]), screen_bin(v[u], scr), tc);
                atomicAdd(&sh[cl * CS + j * W + (y[u] >> 1)], 1u << (16 * (y[u] & 1)));
            }
        }
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    __syncthreads();
    unsigned int* out = part + (size_t)blockIdx.x * gcols * CS;
    for (int i = threadIdx.x; i < words; i += blockDim.x) out[i] = sh[i];
}

// hist[c][j][y] = sum over row ranges of the 16-bit counts (fixed order)
__global__ void __launch_bounds__(kThreads)
k_class_hist_reduce(const unsigned int* __restrict__ part, int d, int nclass, int gcols, int ngroups, int nranges,
                    unsigned int* __restrict__ hist) {
    const int W = (nclass + 1) / 2;
    const int CS = kFine * W + 1;                          // words per column in a block's slot
    const int64_t total = (int64_t)d * kFine * W;
    const size_t slot = (size_t)gcols * CS;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % W);
        const int64_t cj = i / W;                         // c * kFine + j
        const int c = (int)(cj / kFine);
        const int g = c / gcols;
        const size_t inner = (size_t)(c - g * gcols) * CS + (size_t)(cj % kFine) * W + w;
        unsigned int lo = 0, hi = 0;
        for (int rr = 0; rr < nranges; rr++) {
            const unsigned int v = part[((size_t)rr * ngroups + g) * slot + inner];
            lo += v & 0xffffu;
            hi += v >> 16;
        }
        const int y0 = 2 * w;
        hist[cj * nclass + y0] = lo;
        if (y0 + 1 < nclass) hist[cj * nclass + y0 + 1] = hi;
    }
}

// per column (one block): fine-bin counts c_j = sum_y hist[j][y], the quantile
// bin q(j) = floor(B (2 C_j + c_j) / (2 N)), and the joint counts
// n_qy = sum over j with q(j) = q of hist[j][y]
__global__ void __launch_bounds__(1024)
k_quantile_joint(const unsigned int* __restrict__ hist, int64_t N, int B, int nclass,
                 unsigned long long* __restrict__ joint) {
    __shared__ long long part[1024];
    __shared__ unsigned long long sj[kMaxQBins * 4];
    const int c = blockIdx.x;
    const unsigned int* h = hist + (size_t)c * kFine * nclass;
    for (int i = threadIdx.x; i < B * nclass; i += blockDim.x) sj[i] = 0ull;
    constexpr int per = kFine / 1024;
    long long cnt[per];
    long long local = 0;
    for (int k = 0; k < per; k++) {
        const int j = threadIdx.x * per + k;
        long long s = 0;
        for (int y = 0; y < nclass; y++) s += h[(size_t)j * nclass + y];
        cnt[k] = s;
        local += s;
    }
    part[threadIdx.x] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {      // inclusive scan of the thread totals
        const long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long C = part[threadIdx.x] - local;        // count below this thread's first fine bin
    // the thread's bins in order: q(j) is non-decreasing, so counts are summed over a run
    // of equal q and added once per run
    long long qrun = -1;
    unsigned long long run[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k = 0; k < per; k++) {
        const int j = threadIdx.x * per + k;
        long long q = ((long long)B * (2 * C + cnt[k])) / (2 * N);
        if (q > B - 1) q = B - 1;
        if (cnt[k] > 0) {
            if (q != qrun) {
                if (qrun >= 0)
                    for (int y = 0; y < nclass; y++)
                        if (run[y]) atomicAdd(&sj[qrun * nclass + y], run[y]);
                qrun = q;
                for (int y = 0; y < 4; y++) run[y] = 0ull;
            }
            for (int y = 0; y < nclass; y++) run[y] += h[(size_t)j * nclass + y];
        }
        C += cnt[k];
    }
    if (qrun >= 0)
        for (int y = 0; y < nclass; y++)
            if (run[y]) atomicAdd(&sj[qrun * nclass + y], run[y]);
    __syncthreads();
    for (int i = threadIdx.x; i < B * nclass; i += blockDim.x) joint[(size_t)c * B * nclass + i] = sj[i];
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

// column statistics of one call: block partials and the grid
struct ColStats {
    double *pS = nullptr, *pQ = nullptr, *pK = nullptr;
    unsigned long long *pmin = nullptr, *pmax = nullptr;
    int nblk = 0;
    int64_t rows = 0;
};

size_t partial_smem(int d) { return d <= kThreads ? (size_t)(kThreads / d) * d * 16 : 0; }

// Hands out 256-byte aligned pieces of one scratch allocation.  A call lays its
// buffers out twice: once with base == nullptr to learn the total, then over
// the allocation, so each call makes one allocation and one free.
struct Carve {
    unsigned char* base = nullptr;
    size_t off = 0;
    template <typename T>
    void take(T** p, size_t bytes) {
        *p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
    }
};

template <typename Layout>
anova_status carve_all(Scratch& scratch, Layout&& layout) {
    Carve size;
    layout(size);
    Carve c;
    ANOVA_CUDA_TRY(scratch.alloc(&c.base, size.off));
    layout(c);
    return ANOVA_OK;
}

void col_layout(int d, int mode, ColStats& cs, Carve& c) {
    const size_t n = (size_t)cs.nblk * d;
    if (mode == kMoments) {
        c.take(&cs.pS, n * sizeof(double));
        c.take(&cs.pQ, n * sizeof(double));
        c.take(&cs.pK, n * sizeof(double));
    } else {
        c.take(&cs.pmin, n * sizeof(unsigned long long));
        c.take(&cs.pmax, n * sizeof(unsigned long long));
    }
}

// one read of X: mean and sd (kMoments) or lo and hi (kRange) of every column
template <int MODE>
anova_status col_stats(const double* X, int64_t N, int d, int64_t ld, const ColStats& cs, double* out0,
                       double* out1, cudaStream_t st) {
    k_col_partials<MODE><<<cs.nblk, kThreads, partial_smem(d), st>>>(X, N, d, ld, cs.rows, cs.pS, cs.pQ, cs.pK,
                                                                     cs.pmin, cs.pmax);
    k_col_totals<MODE><<<d, kThreads, 0, st>>>(cs.pS, cs.pQ, cs.pK, cs.pmin, cs.pmax, cs.nblk, d, N, cs.rows, out0,
                                               out1);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// per-column thresholds of the fine bins (and their FP32 screens) from one read of X
struct FineBins {
    double *lo = nullptr, *hi = nullptr;
    unsigned long long* thr = nullptr;
    float4* screen = nullptr;
};

void fine_layout(int d, FineBins& fb, Carve& c) {
    c.take(&fb.lo, d * sizeof(double));
    c.take(&fb.hi, d * sizeof(double));
    c.take(&fb.thr, (size_t)d * kThrRow * sizeof(unsigned long long));
    c.take(&fb.screen, d * sizeof(float4));
}

anova_status fine_bins_setup(const double* X, int64_t N, int d, int64_t ld, const ColStats& cs, FineBins& fb,
                             cudaStream_t st) {
    ANOVA_TRY(col_stats<kRange>(X, N, d, ld, cs, fb.lo, fb.hi, st));
    k_fine_thresholds<<<dim3((kThrRow + kThreads - 1) / kThreads, d), kThreads, 0, st>>>(fb.lo, fb.hi, d, fb.thr,
                                                                                         fb.screen);
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
    stat_grid(N, device_sms(), &cs.nblk, &cs.rows);
    ANOVA_TRY(carve_all(scratch, [&](Carve& c) { col_layout(d, kMoments, cs, c); }));
    // one pass: shifted block sums, combined over blocks by the pairwise update
    ANOVA_TRY(col_stats<kMoments>(X, N, d, ld, cs, mean, sd, st));
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
    FineBins fb;
    unsigned long long* joint = nullptr;
    const size_t cells = (size_t)d * bins * nclass;
    stat_grid(N, device_sms(), &cs.nblk, &cs.rows);
    // two passes over X (privatised (fine bin, class) counts) where they fit, else three
    const int W = (nclass + 1) / 2;
    const int sms = device_sms();
    const int gmax = std::max(1, (int)(kCHSmem / (((size_t)kFine * W + 1) * sizeof(unsigned int))));
    const int ngroups = (d + gmax - 1) / gmax;
    const int gcols = (d + ngroups - 1) / ngroups;
    int64_t nranges = std::max<int64_t>((N + kCHMaxRows - 1) / kCHMaxRows,
                                        std::min<int64_t>((2 * sms + ngroups - 1) / ngroups, (N + 4095) / 4096));
    nranges = std::max<int64_t>(nranges, 1);
    const int64_t rows_pb = (N + nranges - 1) / nranges;
    nranges = (N + rows_pb - 1) / rows_pb;
    const size_t slot = (size_t)gcols * (kFine * W + 1);
    const size_t part_bytes = (size_t)nranges * ngroups * slot * sizeof(unsigned int);
    const bool two_pass = nclass <= 4 && part_bytes <= kCHPartMax && nranges * ngroups <= INT32_MAX;
    unsigned int *part = nullptr, *chist = nullptr, *hist = nullptr;
    unsigned char* qmap = nullptr;
    ANOVA_TRY(carve_all(scratch, [&](Carve& c) {
        col_layout(d, kRange, cs, c);
        fine_layout(d, fb, c);
        c.take(&joint, (cells + 1) * sizeof(unsigned long long));
        if (two_pass) {
            c.take(&part, part_bytes);
            c.take(&chist, (size_t)d * kFine * nclass * sizeof(unsigned int));
        } else {
            c.take(&hist, (size_t)d * kFine * sizeof(unsigned int));
            c.take(&qmap, (size_t)d * kFine);
        }
    }));
    unsigned long long* bad = joint + cells;
    ANOVA_TRY(fine_bins_setup(X, N, d, ld, cs, fb, st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(joint, 0, (cells + 1) * sizeof(unsigned long long), st));
    if (two_pass) {
        static bool attr2 = [] {
            cudaFuncSetAttribute(k_fine_class_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCHSmem);
            return true;
        }();
        (void)attr2;
        k_fine_class_hist<<<(unsigned)(nranges * ngroups), kCHThreads, slot * sizeof(unsigned int), st>>>(
            X, N, d, ld, fb.thr, fb.screen, labels, nclass, gcols, ngroups, rows_pb, part, bad);
        k_class_hist_reduce<<<grid_for((int64_t)d * kFine * W, kThreads, 8 * sms), kThreads, 0, st>>>(
            part, d, nclass, gcols, ngroups, (int)nranges, chist);
        k_quantile_joint<<<d, 1024, 0, st>>>(chist, N, bins, nclass, joint);
    } else {
        ANOVA_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)d * kFine * sizeof(unsigned int), st));
        k_fine_hist<<<cs.nblk, kThreads, 0, st>>>(X, N, d, ld, fb.thr, fb.screen, cs.rows, hist);
        k_quantile_map<<<d, 1024, 0, st>>>(hist, N, bins, qmap);
        static bool attr = [] {
            cudaFuncSetAttribute(k_joint, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            return true;
        }();
        (void)attr;
        k_joint<<<cs.nblk, kThreads, cells * sizeof(unsigned int), st>>>(X, N, d, ld, fb.thr, fb.screen, qmap, labels,
                                                                        bins, nclass, cs.rows, joint, bad);
    }
    ANOVA_CHECK_LAUNCH();
    std::vector<unsigned long long> hj(cells + 1);
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

anova_status anova_mis_fine_bins(const double* X, int64_t N, int32_t d, int64_t ld, int32_t* bins, void* stream) {
    if (!shapes_ok(X, N, d, ld) || !bins) {
        set_error("anova_mis_fine_bins: need N >= 1, 1 <= d <= 2048, ld >= d and device pointers");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch scratch(st);
    ColStats cs;
    FineBins fb;
    stat_grid(N, device_sms(), &cs.nblk, &cs.rows);
    ANOVA_TRY(carve_all(scratch, [&](Carve& c) {
        col_layout(d, kRange, cs, c);
        fine_layout(d, fb, c);
    }));
    ANOVA_TRY(fine_bins_setup(X, N, d, ld, cs, fb, st));
    k_fine_bins_out<<<cs.nblk, kThreads, 0, st>>>(X, N, d, ld, fb.thr, fb.screen, cs.rows, bins);
    ANOVA_CHECK_LAUNCH();
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
