// batch.cu -- many kernel ridge regression problems and right-hand sides in
// one launch sequence (the batching form of the paper's fit, Sec. 2 with the
// fast summation of Sec. 4.2 as the operator).
//
// A batch joins P problems (each an FP32 plan of its own nodes, windows,
// width and bandwidths; one cut-off m for all) with R right-hand sides each.
// Every (problem, window, right-hand side) is one "instance": its own grid
// and sorted coefficients, the problem's binned nodes and weight table.  One
// launch per (window dimension, region size) spreads every instance, one
// launch sequence transforms all 3-D grids and one all 1-D / 2-D grids, one
// launch per group gathers.  The P x R conjugate-gradient systems run in
// lockstep on one flat vector space (problem p, right-hand side r, entry i at
// off_p + r N_p + i), FP64 vectors and scalars, per-system step sizes and
// stopping; the iteration is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "common.cuh"

namespace anova {

constexpr int kBChunk = 2048;          // vector entries per block of a system
constexpr int kBThreads = 256;
constexpr int kBCheck = 8;             // iterations per graph replay between host checks

struct BSys {
    double yy, rr, pq, a, b;
    int active, iters;
};

struct BSysInfo {                      // per system, read by the vector kernels
    int64_t off, len;                  // flat offset and length (N_p)
    int64_t tmp;                       // per-window results of window 0 of this system
    int64_t tstride;                   // distance between windows in tmp (R N_p)
    int P, eta_off;                    // windows of the problem and their weights
};

struct SortInst {
    const int32_t* perm;
    float* asort;
    int64_t N, src;                    // nodes; flat offset of the system's coefficients
    const int* live;                   // the system still iterates
};

}  // namespace anova

struct anova_batch {
    int nprob = 0, nrhs = 0, m = 0, sm_count = 1, NS = 0, nchunk = 1, ninst = 0;
    int64_t S = 0;
    std::vector<anova_plan*> plans;
    std::vector<int64_t> off;                      // nprob + 1
    float* grids = nullptr;
    size_t grid_elems = 0;
    float2* work1 = nullptr;
    float2* work2 = nullptr;
    float* asort = nullptr;
    float* tmp = nullptr;
    anova::DenseWin* desc = nullptr;
    int4* sub = nullptr;                           // launch list: sub-problems of the live systems
    int4* sub_full = nullptr;                      // every instance's sub-problems, grouped by (dims, R)
    std::vector<std::array<int, 3>> groups;        // of the launch list
    // host copies for rebuilding the launch lists over the systems still iterating
    struct InstHost { int key, sys, inst, f3, f12; int64_t first, count; };
    std::vector<InstHost> ih;                      // per instance, in sub_full order within a group
    std::vector<int> keys;                         // group keys in launch order
    std::vector<anova::Fft3Win> f3_all;
    std::vector<anova::Fft12Win> f12_all;
    std::vector<anova::SortInst> sort_all;
    int4* copy_tab = nullptr;                      // (src, dst, count) per live instance
    int nsort = 0, live_systems = -1;
    anova::SortInst* sorts = nullptr;
    int64_t max_inst_N = 0;
    anova::Fft3Win* fft3 = nullptr;
    anova::Fft3Shape fft3_shape;
    anova::Fft12Win* fft12 = nullptr;
    int n12 = 0;
    int n12_uniform = -1;                          // shared n of the 1-D / 2-D instances (n_os = 2n), else 0
    size_t smem12 = 0;
    double* eta = nullptr;                         // concatenated window weights
    double* lam = nullptr;                         // per system: lambda of its problem (solve)
    double* zero = nullptr;                        // per system: 0 (matrix-vector product)
    double tol_graph = -1.0;
    int maxit_graph = -1;
    anova::BSysInfo* sys = nullptr;
    anova::BSys* scal = nullptr;
    double* vec = nullptr;                         // x, r, p, q: 4 S
    double* part = nullptr;                        // NS x nchunk partial sums
    int* count = nullptr;                          // active systems
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture = nullptr;
};

namespace anova {

__global__ void k_b_tag(const int4* __restrict__ src, int n, int slot, int4* __restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 v = src[i];
        v.w = slot;
        dst[i] = v;
    }
}

// asort of every instance: the system's coefficients in the window's sorted order, FP32
__global__ void k_b_sort(const SortInst* __restrict__ inst, const double* __restrict__ x) {
    const SortInst s = inst[blockIdx.y];
    if (!*s.live) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.N; i += (int64_t)gridDim.x * blockDim.x)
        s.asort[i] = (float)x[s.src + s.perm[i]];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// x = 0, r = p = y; partial y.y
__global__ void __launch_bounds__(kBThreads)
k_b_init(const BSysInfo* __restrict__ sys, const double* __restrict__ y, double* __restrict__ x,
         double* __restrict__ r, double* __restrict__ p, double* __restrict__ part, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const double v = y[s.off + i];
        x[s.off + i] = 0.0;
        r[s.off + i] = v;
        p[s.off + i] = v;
        acc += v * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

__device__ __forceinline__ double chunk_total(const double* part, int s, int nchunk, int64_t len) {
    const int nc = (int)((len + kBChunk - 1) / kBChunk);
    double t = 0.0;
    for (int c = 0; c < nc; c++) t += part[(size_t)s * nchunk + c];   // fixed order: deterministic
    return t;
}

__global__ void k_b_start(const BSysInfo* __restrict__ sys, BSys* __restrict__ sc, const double* __restrict__ part,
                          int nchunk, int NS) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= NS) return;
    const double yy = chunk_total(part, s, nchunk, sys[s].len);
    BSys v;
    v.yy = yy;
    v.rr = yy;
    v.pq = 0.0;
    v.a = 0.0;
    v.b = 0.0;
    v.active = yy > 0.0 ? 1 : 0;
    v.iters = 0;
    sc[s] = v;
}

// q = sum_l eta_l tmp_l + lambda p; partial p.q (active systems)
__global__ void __launch_bounds__(kBThreads)
k_b_q(const BSysInfo* __restrict__ sys, const BSys* __restrict__ sc, const double* __restrict__ eta,
      const double* __restrict__ lam, const float* __restrict__ tmp, const double* __restrict__ p,
      double* __restrict__ q, double* __restrict__ part, int nchunk, int apply_all) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    if (!apply_all && !sc[blockIdx.y].active) return;
    const double lambda = lam[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        double v = 0.0;
        for (int l = 0; l < s.P; l++) v += eta[s.eta_off + l] * (double)tmp[s.tmp + l * s.tstride + i];
        const double pi = p[s.off + i];
        v += lambda * pi;
        q[s.off + i] = v;
        acc += pi * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

__global__ void k_b_alpha(const BSysInfo* __restrict__ sys, BSys* __restrict__ sc, const double* __restrict__ part,
                          int nchunk, int NS) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= NS || !sc[s].active) return;
    const double pq = chunk_total(part, s, nchunk, sys[s].len);
    sc[s].pq = pq;
    if (pq > 0.0 && isfinite(pq)) {
        sc[s].a = sc[s].rr / pq;
    } else {
        sc[s].a = 0.0;
        sc[s].active = 0;     // breakdown: the system keeps its current iterate
    }
}

// x += a p, r -= a q; partial r.r
__global__ void __launch_bounds__(kBThreads)
k_b_xr(const BSysInfo* __restrict__ sys, const BSys* __restrict__ sc, double* __restrict__ x, double* __restrict__ r,
       const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ part, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    if (!sc[blockIdx.y].active) return;
    const double a = sc[blockIdx.y].a;
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const int64_t e = s.off + i;
        x[e] += a * p[e];
        const double rv = r[e] - a * q[e];
        r[e] = rv;
        acc += rv * rv;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

__global__ void k_b_beta(const BSysInfo* __restrict__ sys, BSys* __restrict__ sc, const double* __restrict__ part,
                         int nchunk, int NS, double tol2, int maxit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= NS || !sc[s].active) return;
    const double rr = chunk_total(part, s, nchunk, sys[s].len);
    BSys v = sc[s];
    v.iters++;
    v.b = rr / v.rr;
    v.rr = rr;
    if (!(rr > tol2 * v.yy) || v.iters >= maxit || !isfinite(rr)) v.active = 0;
    sc[s] = v;
}

// p = r + b p (systems still iterating)
__global__ void __launch_bounds__(kBThreads)
k_b_p(const BSysInfo* __restrict__ sys, const BSys* __restrict__ sc, const double* __restrict__ r,
      double* __restrict__ p) {
    const BSysInfo s = sys[blockIdx.y];
    if (!sc[blockIdx.y].active) return;
    const double b = sc[blockIdx.y].b;
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const int64_t e = s.off + i;
        p[e] = r[e] + b * p[e];
    }
}

__global__ void k_b_live_all(BSys* __restrict__ sc, int NS) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < NS) sc[s].active = 1;
}

__global__ void k_b_count(const BSys* __restrict__ sc, int NS, int* __restrict__ count) {
    __shared__ int c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    int mine = 0;
    for (int s = threadIdx.x; s < NS; s += blockDim.x) mine += sc[s].active;
    atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0) *count = c;
}

// r = y - q; partial r.r (all systems), for the recomputed residual
__global__ void __launch_bounds__(kBThreads)
k_b_resid(const BSysInfo* __restrict__ sys, const double* __restrict__ y, const double* __restrict__ q,
          double* __restrict__ part, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const double d = y[s.off + i] - q[s.off + i];
        acc += d * d;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

__global__ void k_b_totals(const BSysInfo* __restrict__ sys, const double* __restrict__ part, int nchunk, int NS,
                           double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < NS) out[s] = chunk_total(part, s, nchunk, sys[s].len);
}

// r = y - q - lambda x; partial r.r (q = K x in FP64, from the problems' plans)
__global__ void __launch_bounds__(kBThreads)
k_b_refine(const BSysInfo* __restrict__ sys, const double* __restrict__ lam, const double* __restrict__ y,
           const double* __restrict__ q, const double* __restrict__ x, double* __restrict__ r,
           double* __restrict__ part, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const double lambda = lam[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const int64_t e = s.off + i;
        const double v = y[e] - q[e] - lambda * x[e];
        r[e] = v;
        acc += v * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

// partial v.v per system
__global__ void __launch_bounds__(kBThreads)
k_b_norm(const BSysInfo* __restrict__ sys, const double* __restrict__ v, double* __restrict__ part, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const double t = v[s.off + i];
        acc += t * t;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

// w = q + lambda dx = (K + lambda I) dx with q = K dx (FP64); partial r.w and w.w per system
__global__ void __launch_bounds__(kBThreads)
k_b_mr(const BSysInfo* __restrict__ sys, const double* __restrict__ lam, const double* __restrict__ r,
       const double* __restrict__ q, const double* __restrict__ dx, double* __restrict__ w,
       double* __restrict__ part_rw, double* __restrict__ part_ww, int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const double lambda = lam[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double rw = 0.0, ww = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const int64_t e = s.off + i;
        const double v = q[e] + lambda * dx[e];
        w[e] = v;
        rw += r[e] * v;
        ww += v * v;
    }
    rw = block_sum(rw, sh);
    ww = block_sum(ww, sh);
    if (threadIdx.x == 0) {
        part_rw[(size_t)blockIdx.y * nchunk + blockIdx.x] = rw;
        part_ww[(size_t)blockIdx.y * nchunk + blockIdx.x] = ww;
    }
}

// x += t dx, r -= t w for the systems with t != 0; partial r.r per system
__global__ void __launch_bounds__(kBThreads)
k_b_step(const BSysInfo* __restrict__ sys, const double* __restrict__ t, const double* __restrict__ dx,
         const double* __restrict__ w, double* __restrict__ x, double* __restrict__ r, double* __restrict__ part,
         int nchunk) {
    __shared__ double sh[32];
    const BSysInfo s = sys[blockIdx.y];
    const double ts = t[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) {
        const int64_t e = s.off + i;
        double v = r[e];
        if (ts != 0.0) {
            x[e] += ts * dx[e];
            v -= ts * w[e];
            r[e] = v;
        }
        acc += v * v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * nchunk + blockIdx.x] = acc;
}

// partial sums of v.v (one per block) for the power iteration
__global__ void __launch_bounds__(kBThreads) k_dot_partial(const double* __restrict__ v, int64_t n,
                                                           double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += v[i] * v[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// v = scale * w, or (first) a fixed pattern of +-1 and 0.5 entries
__global__ void k_power_next(double* __restrict__ v, const double* __restrict__ w, int64_t n, double scale, int first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = first ? ((i * 2654435761ull) & 4 ? 1.0 : -0.5) : scale * w[i];
}

// y += x over one system's slice
__global__ void k_slice_axpy(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// zero the right-hand side of systems already converged; x += dx for the others
__global__ void __launch_bounds__(kBThreads)
k_b_mask(const BSysInfo* __restrict__ sys, const int* __restrict__ done, double* __restrict__ r) {
    if (!done[blockIdx.y]) return;
    const BSysInfo s = sys[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x) r[s.off + i] = 0.0;
}

__global__ void __launch_bounds__(kBThreads)
k_b_axpy(const BSysInfo* __restrict__ sys, const int* __restrict__ apply, const double* __restrict__ dx,
         double* __restrict__ x, double sign) {
    if (!apply[blockIdx.y]) return;
    const BSysInfo s = sys[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * kBChunk;
    for (int64_t i = lo + threadIdx.x; i < s.len && i < lo + kBChunk; i += blockDim.x)
        x[s.off + i] += sign * dx[s.off + i];
}

__global__ void k_b_copy_subs(const int4* __restrict__ src, const int4* __restrict__ tab, int4* __restrict__ dst) {
    const int4 t = tab[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < t.z; i += gridDim.x * blockDim.x) dst[t.y + i] = src[t.x + i];
}

// Launch lists (sub-problems, FFT descriptors, sort table) over the systems
// with live[s] != 0 only: a stopped system's blocks are not even scheduled.
// The kernels' own live checks cover systems that stop between rebuilds.
static anova_status batch_compact(anova_batch* b, const std::vector<int>& live, cudaStream_t st) {
    std::vector<int4> tab;
    b->groups.clear();
    int at = 0, maxc = 0;
    size_t k = 0;
    for (int key : b->keys) {
        const int first = at;
        for (; k < b->ih.size() && b->ih[k].key == key; k++) {
            const auto& I = b->ih[k];
            if (!live[I.sys] || I.count == 0) continue;
            tab.push_back(make_int4((int)I.first, at, (int)I.count, 0));
            at += (int)I.count;
            maxc = std::max(maxc, (int)I.count);
        }
        if (at > first) b->groups.push_back({key, first, at - first});
    }
    std::vector<Fft3Win> f3;
    std::vector<Fft12Win> f12;
    std::vector<SortInst> so;
    for (const auto& I : b->ih) {
        if (!live[I.sys]) continue;
        if (I.f3 >= 0) f3.push_back(b->f3_all[I.f3]);
        if (I.f12 >= 0) f12.push_back(b->f12_all[I.f12]);
        so.push_back(b->sort_all[I.inst]);
    }
    if (!tab.empty()) {
        ANOVA_CUDA_TRY(cudaMemcpyAsync(b->copy_tab, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        const int gx = std::max(1, std::min((maxc + kThreads - 1) / kThreads, 64));
        k_b_copy_subs<<<dim3(gx, (unsigned)tab.size()), kThreads, 0, st>>>(b->sub_full, b->copy_tab, b->sub);
        ANOVA_CHECK_LAUNCH();
    }
    if (!f3.empty())
        ANOVA_CUDA_TRY(cudaMemcpyAsync(b->fft3, f3.data(), f3.size() * sizeof(Fft3Win), cudaMemcpyHostToDevice, st));
    if (!f12.empty())
        ANOVA_CUDA_TRY(cudaMemcpyAsync(b->fft12, f12.data(), f12.size() * sizeof(Fft12Win), cudaMemcpyHostToDevice, st));
    if (!so.empty())
        ANOVA_CUDA_TRY(cudaMemcpyAsync(b->sorts, so.data(), so.size() * sizeof(SortInst), cudaMemcpyHostToDevice, st));
    // the host vectors are pageable: the copies complete before they return
    b->fft3_shape.nw = (int)f3.size();
    b->n12 = (int)f12.size();
    b->nsort = (int)so.size();
    int nl = 0;
    for (int v : live) nl += v != 0;
    b->live_systems = nl;
    if (b->graph) {                  // launch sizes changed: capture again
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return ANOVA_OK;
}

static anova_status batch_compact_all(anova_batch* b, cudaStream_t st) {
    if (b->live_systems == b->NS) return ANOVA_OK;
    return batch_compact(b, std::vector<int>(b->NS, 1), st);
}

// tmp <- K_l x for every instance (FP32 operator on the FP64 flat vector x)
static anova_status batch_operator(anova_batch* b, const double* x, cudaStream_t st) {
    if (b->nsort == 0) return ANOVA_OK;
    const int gx = (int)std::min<int64_t>((b->max_inst_N + kThreads - 1) / kThreads, 64);
    k_b_sort<<<dim3(gx, b->nsort), kThreads, 0, st>>>(b->sorts, x);
    ANOVA_CHECK_LAUNCH();
    ANOVA_CUDA_TRY(cudaMemsetAsync(b->grids, 0, b->grid_elems * sizeof(float), st));
    ANOVA_TRY(dense_f32_spread_groups(b->m, b->sub, b->desc, b->groups, st,
                                      b->plans[0]->pw12 ? b->plans[0]->psi_host.data() : nullptr,
                                      b->plans[0]->sm_count, b->plans[0]->spread_tc5));
    ANOVA_TRY(fft3_box_run<float>(b->fft3, b->fft3_shape, b->sm_count, st));
    ANOVA_TRY(fft12_box_run<float>(b->fft12, b->n12, b->smem12, st, b->n12_uniform));
    return dense_f32_gather_groups(b->m, b->plans[0]->psi_poly, b->sub, b->desc, b->groups, st,
                                   b->plans[0]->gather_tc5 ? b->plans[0]->psi_host.data() : nullptr,
                                   b->plans[0]->sm_count);
}

static anova_status batch_iteration(anova_batch* b, double tol2, int maxit, cudaStream_t st) {
    double* x = b->vec;
    double* r = x + b->S;
    double* p = r + b->S;
    double* q = p + b->S;
    const dim3 gv(b->nchunk, b->NS);
    const int gs = (b->NS + kBThreads - 1) / kBThreads;
    ANOVA_TRY(batch_operator(b, p, st));
    k_b_q<<<gv, kBThreads, 0, st>>>(b->sys, b->scal, b->eta, b->lam, b->tmp, p, q, b->part, b->nchunk, 0);
    k_b_alpha<<<gs, kBThreads, 0, st>>>(b->sys, b->scal, b->part, b->nchunk, b->NS);
    k_b_xr<<<gv, kBThreads, 0, st>>>(b->sys, b->scal, x, r, p, q, b->part, b->nchunk);
    k_b_beta<<<gs, kBThreads, 0, st>>>(b->sys, b->scal, b->part, b->nchunk, b->NS, tol2, maxit);
    k_b_p<<<gv, kBThreads, 0, st>>>(b->sys, b->scal, r, p);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

}  // namespace anova

using namespace anova;

extern "C" {

void anova_batch_destroy(anova_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->grids);
    cudaFree(b->work1);
    cudaFree(b->work2);
    cudaFree(b->asort);
    cudaFree(b->tmp);
    cudaFree(b->desc);
    cudaFree(b->sub);
    cudaFree(b->sub_full);
    cudaFree(b->copy_tab);
    cudaFree(b->sorts);
    cudaFree(b->fft3);
    cudaFree(b->fft12);
    cudaFree(b->eta);
    cudaFree(b->sys);
    cudaFree(b->scal);
    cudaFree(b->vec);
    cudaFree(b->part);
    cudaFree(b->count);
    cudaFree(b->lam);
    cudaFree(b->zero);
    delete b;
}

anova_status anova_batch_create(anova_plan* const* plans, int32_t nprob, int32_t nrhs, void* stream,
                                anova_batch** out) {
    if (!out || !plans || nprob < 1 || nrhs < 1 || (int64_t)nprob * nrhs > 65535) {
        set_error("anova_batch_create: need 1 <= problems x right-hand sides <= 65535 and valid pointers");
        return ANOVA_EINVAL;
    }
    *out = nullptr;
    for (int p = 0; p < nprob; p++) {
        const anova_plan* pl = plans[p];
        if (!pl || !(pl->precision & ANOVA_FP32) || pl->N < 1 || pl->m != plans[0]->m ||
            pl->sigma != plans[0]->sigma) {
            set_error("anova_batch_create: every plan must hold FP32, have nodes and share the cut-off m and sigma");
            return ANOVA_EINVAL;
        }
        for (int l = 0; l < pl->P; l++) {
            const WindowPlan& w = pl->win[l];
            const bool weights = w.wtab || (w.dA < 3 && pl->pw12 && tc5_supported(w.R, pl->m));
            if (!w.dense || !weights || !(w.dA == 3 ? fft3_box_supported(w) : w.fft12)) {
                set_error("anova_batch_create: problem " + std::to_string(p) + " window " + std::to_string(l) +
                          " is not on the dense kernels and box FFTs");
                return ANOVA_EINVAL;
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    anova_batch* b = new (std::nothrow) anova_batch();
    if (!b) return ANOVA_ENOMEM;
    b->nprob = nprob;
    b->nrhs = nrhs;
    b->m = plans[0]->m;
    b->sm_count = plans[0]->sm_count;
    b->plans.assign(plans, plans + nprob);
    b->off.assign(nprob + 1, 0);
    int64_t maxN = 0;
    for (int p = 0; p < nprob; p++) {
        b->off[p + 1] = b->off[p] + plans[p]->N * nrhs;
        maxN = std::max(maxN, plans[p]->N);
    }
    b->S = b->off[nprob];
    b->NS = nprob * nrhs;
    b->nchunk = (int)((maxN + kBChunk - 1) / kBChunk);

    // instances (p, l, r) in this order; per-instance grid, work, asort, tmp offsets
    struct Inst { int p, l, r; size_t grid, work; int64_t as, tmp; };
    std::vector<Inst> inst;
    size_t grid_elems = 0, work_elems = 0;
    int64_t as_elems = 0, tmp_elems = 0;
    std::vector<int64_t> tmp_base(nprob);
    for (int p = 0; p < nprob; p++) {
        const anova_plan* pl = plans[p];
        tmp_base[p] = tmp_elems;
        for (int l = 0; l < pl->P; l++) {
            const WindowPlan& w = pl->win[l];
            size_t ge = 1;
            for (int t = 0; t < w.dA; t++) ge *= w.nos;
            ge = (ge + 63) & ~(size_t)63;
            const size_t we = w.dA == 3 ? (((size_t)w.nos * w.nos * w.n + 31) & ~(size_t)31) : 0;
            for (int r = 0; r < nrhs; r++) {
                inst.push_back({p, l, r, grid_elems, work_elems, as_elems, tmp_elems});
                grid_elems += ge;
                work_elems += we;
                as_elems += pl->N;
                tmp_elems += pl->N;
            }
        }
    }
    if (inst.size() > 65535) {
        set_error("anova_batch_create: more than 65535 (problem, window, right-hand side) instances");
        delete b;
        return ANOVA_EINVAL;
    }
    b->ninst = (int)inst.size();
    b->grid_elems = grid_elems;
    anova_status s = ANOVA_OK;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (s == ANOVA_OK && anova::dev_malloc((void**)ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            set_error("anova_batch_create: out of device memory");
            s = ANOVA_ENOMEM;
        }
    };
    alloc((void**)&b->grids, grid_elems * sizeof(float));
    alloc((void**)&b->work1, work_elems * sizeof(float2));
    alloc((void**)&b->work2, work_elems * sizeof(float2));
    alloc((void**)&b->asort, as_elems * sizeof(float));
    alloc((void**)&b->tmp, tmp_elems * sizeof(float));
    alloc((void**)&b->vec, 4 * b->S * sizeof(double));
    alloc((void**)&b->part, (size_t)b->NS * b->nchunk * sizeof(double));
    alloc((void**)&b->scal, (size_t)b->NS * sizeof(BSys));
    alloc((void**)&b->sys, (size_t)b->NS * sizeof(BSysInfo));
    alloc((void**)&b->count, sizeof(int));
    alloc((void**)&b->lam, (size_t)b->NS * sizeof(double));
    alloc((void**)&b->zero, (size_t)b->NS * sizeof(double));
    if (s != ANOVA_OK) {
        anova_batch_destroy(b);
        return s;
    }

    // dense descriptors, sort table, FFT descriptors
    std::vector<DenseWin> desc(inst.size());
    std::vector<SortInst> sorts(inst.size());
    std::vector<Fft3Win> f3;
    std::vector<Fft12Win> f12;
    for (size_t k = 0; k < inst.size(); k++) {
        const Inst& I = inst[k];
        const anova_plan* pl = plans[I.p];
        const WindowPlan& w = pl->win[I.l];
        DenseWin& d = desc[k];
        d.perm = w.X.perm;
        d.cell = w.X.cell;
        d.frac = w.X.frac32;
        d.wtab = w.wtab;
        d.asort = b->asort + I.as;
        d.grid = b->grids + I.grid;
        d.out = b->tmp + I.tmp;
        d.N = pl->N;
        d.nos = w.nos;
        d.Tb = w.T;
        d.nb = w.nb;
        d.pad = 0;
        const int* live = &b->scal[I.p * nrhs + I.r].active;
        d.live = live;
        sorts[k] = {w.X.perm, b->asort + I.as, pl->N, b->off[I.p] + (int64_t)I.r * pl->N, live};
        b->max_inst_N = std::max(b->max_inst_N, pl->N);
        if (w.dA == 3) {
            Fft3Win f;
            f.grid = b->grids + I.grid;
            f.buf1 = b->work1 + I.work;
            f.buf2 = b->work2 + I.work;
            f.tw = w.tw32;
            f.D = w.D32;
            for (int t = 0; t < 3; t++) {
                f.lo[t] = w.box_lo[t];
                f.B[t] = w.box_ext[t];
            }
            f.n = w.n;
            f.nos = w.nos;
            f.live = live;
            f3.push_back(f);
            b->fft3_shape.add(w);
        } else {
            Fft12Win f;
            f.grid = b->grids + I.grid;
            f.tw = w.tw32;
            f.D = w.D32;
            f.dA = w.dA;
            f.n = w.n;
            f.nos = w.nos;
            for (int t = 0; t < 2; t++) {
                f.lo[t] = w.box_lo[t];
                f.B[t] = w.box_ext[t];
            }
            f.live = live;
            f12.push_back(f);
            const int un = w.nos == 2 * w.n ? w.n : 0;
            b->n12_uniform = (b->n12_uniform < 0) ? un : (b->n12_uniform == un ? un : 0);
            b->smem12 = std::max(b->smem12, fft12_window_smem(w, sizeof(float)));
        }
    }
    b->n12 = (int)f12.size();
    // merged sub-problem list grouped by (dims, region size)
    std::map<int, std::vector<int>> by_key;
    int64_t total_sub = 0;
    for (size_t k = 0; k < inst.size(); k++) {
        const WindowPlan& w = plans[inst[k].p]->win[inst[k].l];
        by_key[w.dA * 100 + w.R].push_back((int)k);
        total_sub += w.X.nsub;
    }
    if (total_sub > INT32_MAX) {
        set_error("anova_batch_create: too many sub-problems");
        anova_batch_destroy(b);
        return ANOVA_EINVAL;
    }
    alloc((void**)&b->sub, total_sub * sizeof(int4));
    alloc((void**)&b->sub_full, total_sub * sizeof(int4));
    alloc((void**)&b->copy_tab, inst.size() * sizeof(int4));
    alloc((void**)&b->desc, desc.size() * sizeof(DenseWin));
    alloc((void**)&b->sorts, sorts.size() * sizeof(SortInst));
    alloc((void**)&b->fft3, f3.size() * sizeof(Fft3Win));
    alloc((void**)&b->fft12, f12.size() * sizeof(Fft12Win));
    if (s != ANOVA_OK) {
        anova_batch_destroy(b);
        return s;
    }
    int at = 0;
    {
        std::vector<int> f3_of(inst.size(), -1), f12_of(inst.size(), -1);
        int c3 = 0, c12 = 0;
        for (size_t k = 0; k < inst.size(); k++) {
            if (plans[inst[k].p]->win[inst[k].l].dA == 3) f3_of[k] = c3++;
            else f12_of[k] = c12++;
        }
        for (const auto& kv : by_key) {
            b->keys.push_back(kv.first);
            for (int k : kv.second) {
                const WindowPlan& w = plans[inst[k].p]->win[inst[k].l];
                b->ih.push_back({kv.first, inst[k].p * nrhs + inst[k].r, k, f3_of[k], f12_of[k], at, w.X.nsub});
                if (w.X.nsub == 0) continue;
                k_b_tag<<<grid_for(w.X.nsub, kThreads, 256), kThreads, 0, st>>>(w.X.sub, w.X.nsub, k,
                                                                               b->sub_full + at);
                at += w.X.nsub;
            }
        }
    }
    b->f3_all = f3;
    b->f12_all = f12;
    b->sort_all = sorts;
    // per-system data and weights
    std::vector<BSysInfo> sys(b->NS);
    std::vector<double> eta;
    for (int p = 0; p < nprob; p++) {
        const anova_plan* pl = plans[p];
        const int eoff = (int)eta.size();
        for (int l = 0; l < pl->P; l++) eta.push_back(pl->win[l].eta);
        for (int r = 0; r < nrhs; r++) {
            BSysInfo& v = sys[p * nrhs + r];
            v.off = b->off[p] + (int64_t)r * pl->N;
            v.len = pl->N;
            v.tmp = tmp_base[p] + (int64_t)r * pl->N;
            v.tstride = (int64_t)nrhs * pl->N;
            v.P = pl->P;
            v.eta_off = eoff;
        }
    }
    alloc((void**)&b->eta, eta.size() * sizeof(double));
    if (s != ANOVA_OK) {
        anova_batch_destroy(b);
        return s;
    }
    cudaError_t e = cudaMemcpyAsync(b->desc, desc.data(), desc.size() * sizeof(DenseWin), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->sorts, sorts.data(), sorts.size() * sizeof(SortInst), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !f3.empty())
        e = cudaMemcpyAsync(b->fft3, f3.data(), f3.size() * sizeof(Fft3Win), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !f12.empty())
        e = cudaMemcpyAsync(b->fft12, f12.data(), f12.size() * sizeof(Fft12Win), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->sys, sys.data(), sys.size() * sizeof(BSysInfo), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->eta, eta.data(), eta.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->zero, 0, (size_t)b->NS * sizeof(double), st);
    if (e == cudaSuccess && batch_compact_all(b, st) != ANOVA_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error(std::string("anova_batch_create: ") + cudaGetErrorString(e));
        anova_batch_destroy(b);
        return ANOVA_ECUDA;
    }
    *out = b;
    return ANOVA_OK;
}

anova_status anova_batch_layout(const anova_batch* b, int64_t* offsets) {
    if (!b || !offsets) return ANOVA_EINVAL;
    for (int p = 0; p <= b->nprob; p++) offsets[p] = b->off[p];
    return ANOVA_OK;
}

anova_status anova_batch_matvec(anova_batch* b, const double* x, double* y, void* stream) {
    if (!b || !x || !y || x == y) {
        set_error("anova_batch_matvec: bad batch or vectors (y must not alias x)");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_b_live_all<<<(b->NS + kBThreads - 1) / kBThreads, kBThreads, 0, st>>>(b->scal, b->NS);
    ANOVA_TRY(batch_compact_all(b, st));
    ANOVA_TRY(batch_operator(b, x, st));
    k_b_q<<<dim3(b->nchunk, b->NS), kBThreads, 0, st>>>(b->sys, b->scal, b->eta, b->zero, b->tmp, x, y, b->part,
                                                        b->nchunk, 1);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

static anova_status batch_cg_solve(anova_batch* b, const double* lambda, const double* y, double* alpha, double tol,
                                   int32_t maxit, int32_t* iters, double* relres, void* stream) {
    if (!b || !lambda || !y || !alpha || y == alpha || !(tol > 0.0) || maxit < 1) {
        set_error("krr_batch_cg_solve: bad batch, lambda, vectors, tol or maxit");
        return ANOVA_EINVAL;
    }
    for (int p = 0; p < b->nprob; p++)
        if (!(lambda[p] >= 0.0)) {
            set_error("krr_batch_cg_solve: lambda must be >= 0");
            return ANOVA_EINVAL;
        }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> lam(b->NS);
    for (int s = 0; s < b->NS; s++) lam[s] = lambda[s / b->nrhs];
    ANOVA_CUDA_TRY(cudaMemcpyAsync(b->lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    double* x = b->vec;
    double* r = x + b->S;
    double* p = r + b->S;
    double* q = p + b->S;
    const dim3 gv(b->nchunk, b->NS);
    const int gs = (b->NS + kBThreads - 1) / kBThreads;
    k_b_init<<<gv, kBThreads, 0, st>>>(b->sys, y, x, r, p, b->part, b->nchunk);
    k_b_start<<<gs, kBThreads, 0, st>>>(b->sys, b->scal, b->part, b->nchunk, b->NS);
    ANOVA_CHECK_LAUNCH();
    const double tol2 = tol * tol;
    // one block of kBCheck iterations per replay; the first block runs directly
    // (one-time kernel attributes are set outside any capture), the second
    // captures the graph for this (tol, maxit)
    if (b->graph && (b->tol_graph != tol || b->maxit_graph != maxit)) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    std::vector<BSys> hs(b->NS);
    std::vector<int> live(b->NS);
    auto recompact = [&]() -> anova_status {
        ANOVA_CUDA_TRY(cudaMemcpyAsync(hs.data(), b->scal, b->NS * sizeof(BSys), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        for (int k = 0; k < b->NS; k++) live[k] = hs[k].active;
        return batch_compact(b, live, st);
    };
    ANOVA_TRY(recompact());
    int done = 0, blocks = 0;
    int active = b->live_systems;
    while (done < maxit && active > 0) {
        if (active <= (3 * b->live_systems) / 4) ANOVA_TRY(recompact());   // drop stopped systems' launches
        if (b->graph) {
            ANOVA_CUDA_TRY(cudaGraphLaunch(b->graph, st));
        } else if (blocks == 0) {
            for (int k = 0; k < kBCheck; k++) ANOVA_TRY(batch_iteration(b, tol2, maxit, st));
        } else {
            if (!b->capture) ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
            ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
            cudaGraph_t g = nullptr;
            ANOVA_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
            anova_status cs = ANOVA_OK;
            for (int k = 0; k < kBCheck && cs == ANOVA_OK; k++) cs = batch_iteration(b, tol2, maxit, b->capture);
            cudaError_t ce = cudaStreamEndCapture(b->capture, &g);
            if (cs != ANOVA_OK) {
                if (g) cudaGraphDestroy(g);
                return cs;
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                set_error(std::string("krr_batch_cg_solve: graph: ") + cudaGetErrorString(ce));
                return ANOVA_ECUDA;
            }
            b->tol_graph = tol;
            b->maxit_graph = maxit;
            ANOVA_CUDA_TRY(cudaGraphLaunch(b->graph, st));
        }
        done += kBCheck;
        blocks++;
        k_b_count<<<1, 1024, 0, st>>>(b->scal, b->NS, b->count);
        ANOVA_CHECK_LAUNCH();
        ANOVA_CUDA_TRY(cudaMemcpyAsync(&active, b->count, sizeof(int), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ANOVA_CUDA_TRY(cudaMemcpyAsync(alpha, x, b->S * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // recomputed residual ||y - (K + lambda I) alpha|| / ||y|| with the batch's operator
    std::vector<BSys> sc(b->NS);
    ANOVA_CUDA_TRY(cudaMemcpyAsync(sc.data(), b->scal, b->NS * sizeof(BSys), cudaMemcpyDeviceToHost, st));
    k_b_live_all<<<gs, kBThreads, 0, st>>>(b->scal, b->NS);
    ANOVA_TRY(batch_compact_all(b, st));
    ANOVA_TRY(batch_operator(b, alpha, st));
    k_b_q<<<gv, kBThreads, 0, st>>>(b->sys, b->scal, b->eta, b->lam, b->tmp, alpha, q, b->part, b->nchunk, 1);
    k_b_resid<<<gv, kBThreads, 0, st>>>(b->sys, y, q, b->part, b->nchunk);
    k_b_totals<<<gs, kBThreads, 0, st>>>(b->sys, b->part, b->nchunk, b->NS, r);
    ANOVA_CHECK_LAUNCH();
    std::vector<double> rr(b->NS);
    ANOVA_CUDA_TRY(cudaMemcpyAsync(rr.data(), r, b->NS * sizeof(double), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    bool all = true;
    for (int s = 0; s < b->NS; s++) {
        const double rel = sc[s].yy > 0.0 ? std::sqrt(rr[s] / sc[s].yy) : 0.0;
        if (iters) iters[s] = sc[s].iters;
        if (relres) relres[s] = rel;     // NaN / inf for a system that broke down
        if (!(sc[s].rr <= tol2 * sc[s].yy) || !std::isfinite(rel)) all = false;
    }
    if (!all) set_error("krr_batch_cg_solve: some systems stopped before reaching tol (see relres)");
    return all ? ANOVA_OK : ANOVA_ENOCONV;
}

// lambda_max of a problem's FP64 kernel matrix by 20 power iterations; v, w:
// device work vectors of the problem's N entries, part: at least 64 doubles
static anova_status power_lambda_max(anova_plan* plan, double* v, double* w, double* part, double* out,
                                     cudaStream_t st) {
    const int64_t n = plan->N;
    *out = 0.0;
    if (n == 0) return ANOVA_OK;
    const int nb = (int)std::min<int64_t>(64, (n + kBThreads - 1) / kBThreads);
    auto norm = [&](const double* x, double* r) -> anova_status {
        k_dot_partial<<<nb, kBThreads, 0, st>>>(x, n, part);
        ANOVA_CHECK_LAUNCH();
        double h[64];
        ANOVA_CUDA_TRY(cudaMemcpyAsync(h, part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        double t = 0.0;
        for (int i = 0; i < nb; i++) t += h[i];
        *r = std::sqrt(t);
        return ANOVA_OK;
    };
    k_power_next<<<nb, kBThreads, 0, st>>>(v, nullptr, n, 1.0, 1);
    double nv = 0.0;
    ANOVA_TRY(norm(v, &nv));
    for (int it = 0; it < 20 && nv > 0.0; it++) {
        ANOVA_TRY(anova_matvec(plan, ANOVA_FP64, v, w, 1, n, st));
        double nw = 0.0;
        ANOVA_TRY(norm(w, &nw));
        *out = nw / nv;
        if (!(nw > 0.0)) break;
        k_power_next<<<nb, kBThreads, 0, st>>>(v, w, n, 1.0 / nw, 0);
        nv = 1.0;
    }
    return ANOVA_OK;
}

static anova_status batch_cg_solve_refined(anova_batch* b, const double* lambda, const double* y, double* alpha,
                                           double tol, int32_t maxit, int32_t* iters, double* relres, void* stream) {
    if (!b || !lambda || !y || !alpha || y == alpha || !(tol > 0.0) || maxit < 1) {
        set_error("krr_batch_cg_solve_refined: bad batch, lambda, vectors, tol or maxit");
        return ANOVA_EINVAL;
    }
    for (const anova_plan* pl : b->plans)
        if (!(pl->precision & ANOVA_FP64)) {
            set_error("krr_batch_cg_solve_refined: every plan must hold FP64 as well (ANOVA_MIXED)");
            return ANOVA_EINVAL;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 gv(b->nchunk, b->NS);
    const int gs = (b->NS + kBThreads - 1) / kBThreads;
    const int NS = b->NS;
    // scratch: allocated together, freed together on every exit
    double *q = nullptr, *r = nullptr, *rin = nullptr, *dx = nullptr, *w = nullptr, *tot = nullptr, *tdev = nullptr,
           *part2 = nullptr;
    int* done = nullptr;
    anova_status s = ANOVA_OK;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (s == ANOVA_OK && anova::dev_malloc_async((void**)ptr, bytes, st) != cudaSuccess) {
            set_error("krr_batch_cg_solve_refined: out of device memory for the solver's vectors");
            s = ANOVA_ENOMEM;
        }
    };
    alloc((void**)&q, b->S * sizeof(double));
    alloc((void**)&r, b->S * sizeof(double));
    alloc((void**)&rin, b->S * sizeof(double));
    alloc((void**)&dx, b->S * sizeof(double));
    alloc((void**)&w, b->S * sizeof(double));
    alloc((void**)&tot, std::max(2 * NS, 64) * sizeof(double));
    alloc((void**)&tdev, NS * sizeof(double));
    alloc((void**)&part2, (size_t)NS * b->nchunk * sizeof(double));
    alloc((void**)&done, NS * sizeof(int));
    std::vector<double> lam(NS), yy(NS), rr(NS), rw(NS), ww(NS), t(NS);
    std::vector<int> conv(NS, 0), stalled(NS, 0), total_it(NS, 0), it(NS, 0), closed(NS, 0);
    std::vector<double> inner_rel(NS);
    for (int k = 0; k < NS; k++) lam[k] = lambda[k / b->nrhs];
    auto totals = [&](const double* prt, std::vector<double>& out) -> anova_status {
        k_b_totals<<<gs, kBThreads, 0, st>>>(b->sys, prt, b->nchunk, NS, tot);
        ANOVA_CHECK_LAUNCH();
        ANOVA_CUDA_TRY(cudaMemcpyAsync(out.data(), tot, NS * sizeof(double), cudaMemcpyDeviceToHost, st));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
        return ANOVA_OK;
    };
    // q = K64 v for every system (each problem's FP64 operator on its right-hand sides)
    auto apply64 = [&](const double* v, double* out) -> anova_status {
        for (int p = 0; p < b->nprob; p++)
            ANOVA_TRY(anova_matvec(b->plans[p], ANOVA_FP64, v + b->off[p], out + b->off[p], b->nrhs,
                                   b->plans[p]->N, stream));
        return ANOVA_OK;
    };
    // r = y - (K64 + lambda I) x from scratch, rr = r.r
    auto true_residuals = [&]() -> anova_status {
        ANOVA_TRY(apply64(alpha, q));
        k_b_refine<<<gv, kBThreads, 0, st>>>(b->sys, b->lam, y, q, alpha, r, b->part, b->nchunk);
        ANOVA_CHECK_LAUNCH();
        return totals(b->part, rr);
    };
    if (s == ANOVA_OK &&
        (cudaMemcpyAsync(b->lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemsetAsync(alpha, 0, b->S * sizeof(double), st) != cudaSuccess ||
         cudaMemcpyAsync(r, y, b->S * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)) {
        set_error("krr_batch_cg_solve_refined: setup copy failed");
        s = ANOVA_ECUDA;
    }
    if (s == ANOVA_OK) {
        k_b_norm<<<gv, kBThreads, 0, st>>>(b->sys, y, b->part, b->nchunk);
        s = totals(b->part, yy);
        rr = yy;
    }
    // Passes: the batched FP32 CG on the current FP64 residual gives a correction
    // dx; the step t dx with t minimising the FP64 residual ||r - t (K64 + lambda I) dx||
    // is taken (never raising it).  A system whose residual norm falls by less than
    // 10 % in a pass has outrun what its FP32 operator resolves: it leaves the
    // batched passes for plain FP64 CG on its correction equation.
    const int kMaxPass = 40;
    for (int pass = 0; s == ANOVA_OK && pass < kMaxPass; pass++) {
        bool any_open = false;
        double worst = 0.0;
        for (int k = 0; k < NS; k++) {
            const double rel = yy[k] > 0.0 ? std::sqrt(rr[k] / yy[k]) : 0.0;
            if (!std::isfinite(rel)) {
                set_error("krr_batch_cg_solve_refined: non-finite residual in system " + std::to_string(k));
                s = ANOVA_ERANGE;
                break;
            }
            conv[k] = rel <= tol;
            closed[k] = conv[k] || stalled[k] || total_it[k] >= maxit;
            if (!closed[k]) {
                any_open = true;
                worst = std::max(worst, rel);
            }
        }
        if (s != ANOVA_OK || !any_open) break;
        if (cudaMemcpyAsync(rin, r, b->S * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(done, closed.data(), NS * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            s = ANOVA_ECUDA;
            break;
        }
        k_b_mask<<<gv, kBThreads, 0, st>>>(b->sys, done, rin);
        // relative to this pass's residual: 1e-4 (about what the FP32 operator
        // resolves), or only what is left to the target when that is less
        const double inner = std::min(0.5, std::max(1e-4, 0.5 * tol / std::max(worst, 1e-300)));
        // at most maxit / 8 inner iterations per pass, so that a system the FP32
        // operator cannot resolve stalls early and keeps budget for the fallback
        const int inner_maxit = std::max(64, maxit / 8);
        s = krr_batch_cg_solve(b, lambda, rin, dx, inner, inner_maxit, it.data(), inner_rel.data(), stream);
        if (s == ANOVA_ENOCONV) s = ANOVA_OK;
        if (s != ANOVA_OK) break;
        if ((s = apply64(dx, q)) != ANOVA_OK) break;
        k_b_mr<<<gv, kBThreads, 0, st>>>(b->sys, b->lam, r, q, dx, w, b->part, part2, b->nchunk);
        if ((s = totals(b->part, rw)) != ANOVA_OK || (s = totals(part2, ww)) != ANOVA_OK) break;
        for (int k = 0; k < NS; k++) {
            t[k] = 0.0;
            if (closed[k]) continue;
            total_it[k] += it[k];
            if (std::isfinite(inner_rel[k]) && std::isfinite(rw[k]) && ww[k] > 0.0) t[k] = rw[k] / ww[k];
        }
        if (cudaMemcpyAsync(tdev, t.data(), NS * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            s = ANOVA_ECUDA;
            break;
        }
        const std::vector<double> rr_old = rr;
        k_b_step<<<gv, kBThreads, 0, st>>>(b->sys, tdev, dx, w, alpha, r, b->part, b->nchunk);
        if ((s = totals(b->part, rr)) != ANOVA_OK) break;
        for (int k = 0; k < NS; k++)
            if (!closed[k] && !(rr[k] <= 0.81 * rr_old[k])) stalled[k] = 1;
    }
    // the recursive residual drifts from the true one: recompute it
    if (s == ANOVA_OK) s = true_residuals();
    // plain FP64 CG on the correction equation of every system still above tol
    // that it can bring to tol within the remaining budget: CG needs about
    // 0.5 sqrt(kappa) ln(2 / eps) iterations to reduce the error by eps, with
    // kappa = (lambda_max(K) + lambda) / lambda and lambda_max(K) from 20 power
    // iterations of the problem's FP64 operator
    bool fallback = false;
    std::vector<double> lmax(b->nprob, -1.0);
    for (int k = 0; s == ANOVA_OK && k < NS; k++) {
        const double rel = yy[k] > 0.0 ? std::sqrt(rr[k] / yy[k]) : 0.0;
        if (rel <= tol || total_it[k] >= maxit) continue;
        const int p = k / b->nrhs;
        const int64_t o = b->off[p] + (int64_t)(k % b->nrhs) * b->plans[p]->N;
        if (lmax[p] < 0.0) {
            s = power_lambda_max(b->plans[p], dx + o, w + o, tot, &lmax[p], st);
            if (s != ANOVA_OK) break;
        }
        const double kappa = (lmax[p] + lam[k]) / lam[k];
        const double need = 0.5 * std::sqrt(kappa) * std::log(2.0 * rel / tol);
        if (need > (double)(maxit - total_it[k])) continue;   // beyond the budget: left as it is
        int itc = 0;
        double relc = 0.0;
        s = cg_fp64_solve(b->plans[p], lam[k], r + o, dx + o, std::min(0.5, tol / rel), maxit - total_it[k], &itc,
                          &relc, st);
        if (s != ANOVA_OK) break;
        total_it[k] += itc;
        k_slice_axpy<<<grid_for(b->plans[p]->N, kBThreads, 8 * b->sm_count), kBThreads, 0, st>>>(
            b->plans[p]->N, dx + o, alpha + o);
        fallback = true;
    }
    if (s == ANOVA_OK && fallback) s = true_residuals();
    bool all = s == ANOVA_OK;
    for (int k = 0; k < NS; k++) {
        const double rel = yy[k] > 0.0 ? std::sqrt(rr[k] / yy[k]) : 0.0;
        if (relres) relres[k] = rel;
        if (iters) iters[k] = total_it[k];
        if (!(rel <= tol)) all = false;
    }
    cudaFreeAsync(q, st);
    cudaFreeAsync(r, st);
    cudaFreeAsync(rin, st);
    cudaFreeAsync(dx, st);
    cudaFreeAsync(w, st);
    cudaFreeAsync(tot, st);
    cudaFreeAsync(tdev, st);
    cudaFreeAsync(part2, st);
    cudaFreeAsync(done, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == ANOVA_OK && e != cudaSuccess) {
        set_error(std::string("krr_batch_cg_solve_refined: ") + cudaGetErrorString(e));
        s = ANOVA_ECUDA;
    }
    if (s != ANOVA_OK) return s;
    return all ? ANOVA_OK : ANOVA_ENOCONV;
}

// The synchronous solves report ETIMEOUT when a bounded wait inside one of
// their kernels gave up (the device counter moved during the call).
anova_status krr_batch_cg_solve(anova_batch* b, const double* lambda, const double* y, double* alpha, double tol,
                                int32_t maxit, int32_t* iters, double* relres, void* stream) {
    const uint64_t w0 = wait_timeouts_on((cudaStream_t)stream);
    const anova_status s = batch_cg_solve(b, lambda, y, alpha, tol, maxit, iters, relres, stream);
    return waits_moved(w0, (cudaStream_t)stream, "krr_batch_cg_solve", s);
}

anova_status krr_batch_cg_solve_refined(anova_batch* b, const double* lambda, const double* y, double* alpha,
                                        double tol, int32_t maxit, int32_t* iters, double* relres, void* stream) {
    const uint64_t w0 = wait_timeouts_on((cudaStream_t)stream);
    const anova_status s = batch_cg_solve_refined(b, lambda, y, alpha, tol, maxit, iters, relres, stream);
    return waits_moved(w0, (cudaStream_t)stream, "krr_batch_cg_solve_refined", s);
}

}  // extern "C"
