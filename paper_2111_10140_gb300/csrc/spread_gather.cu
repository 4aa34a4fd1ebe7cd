// spread_gather.cu -- window steps of the adjoint NFFT and of the NFFT
// (arXiv 2111.10140, Sec. 4.1 Eq. adjnfft / Eq. nfft, used by the fast
// summation of Sec. 4.2 Eq. fastsum).
//
//   spread:  g_u = sum_j alpha_j prod_t psi(nos x_{j,t} - u_t)
//   gather:  s_i = sum_u h_u prod_t psi(nos z_{i,t} - u_t)
//
// psi is the Kaiser-Bessel window normalised to psi(0) = 1, nonzero for
// |t| <= m, so each node touches 2m+1 grid cells per axis: u = c - m .. c + m
// for the node's cell c (the tap c + m + 1 always has |t| > m).
//
// Nodes are sorted by bins of T^dA cells.  One CTA handles one sub-problem
// (one bin, at most kSubChunk nodes); all its taps fall in the region of
// R = T + 2m cells per axis starting at cell (bin * T - m), which lives in
// shared memory.  Spreading accumulates the region with shared atomics and
// adds it to the global grid once; gathering stages the region once and
// reads all taps from shared memory.
#include <cuda_runtime.h>

#include "common.cuh"

namespace anova {

template <typename T, int DA>
__device__ __forceinline__ void bin_coords(int bin, int nb, int* bc) {
    for (int t = DA - 1; t >= 0; t--) {
        bc[t] = bin % nb;
        bin /= nb;
    }
}

template <typename T, int DA>
__device__ __forceinline__ int region_to_grid(int i, int R, const int* bc, int Tb, int m, int nos) {
    int rr[3];
    for (int t = DA - 1; t >= 0; t--) {
        rr[t] = i % R;
        i /= R;
    }
    int g = 0;
    for (int t = 0; t < DA; t++) {
        int u = bc[t] * Tb - m + rr[t];
        u %= nos;
        if (u < 0) u += nos;
        g = g * nos + u;
    }
    return g;
}

// taps w[t][k] = psi(m - k + f_t) of a node; from the plan's FP64 tap table when
// given (the plan's own nodes in an FP64 plan), else evaluated
template <typename T, int DA>
__device__ __forceinline__ void node_weights(const int32_t* __restrict__ cell, const T* __restrict__ frac,
                                             int64_t N, int64_t pos, const int* bc, int Tb, int m,
                                             T b, T norm, const double* __restrict__ tap, T (*w)[2 * kMaxM + 1],
                                             int* off) {
    const T mm = (T)m;
    for (int t = 0; t < DA; t++) {
        off[t] = cell[t * N + pos] - bc[t] * Tb;
        if (tap) {
            const double* tp = tap + (pos * DA + t) * (2 * m + 1);
            for (int k = 0; k <= 2 * m; k++) w[t][k] = (T)tp[k];
        } else {
            const T f = frac[t * N + pos];
            for (int k = 0; k <= 2 * m; k++) w[t][k] = kb_psi<T>(f + mm - (T)k, mm, b, norm);
        }
    }
}

template <typename T, int DA>
__global__ void __launch_bounds__(kThreads)
k_spread(const int4* __restrict__ sub, const int32_t* __restrict__ perm, const int32_t* __restrict__ cell,
         const T* __restrict__ frac, int64_t N, const void* __restrict__ alpha, int alpha_double,
         T* __restrict__ grid, int nos, int Tb, int nb, int R, int m, T b, T norm, const double* __restrict__ tap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);
    const int4 sp = sub[blockIdx.x];
    int bc[3] = {0, 0, 0};
    bin_coords<T, DA>(sp.x, nb, bc);
    int RD = R;
    if (DA > 1) RD *= R;
    if (DA > 2) RD *= R;
    for (int i = threadIdx.x; i < RD; i += blockDim.x) acc[i] = T(0);
    __syncthreads();
    const int ntap = 2 * m + 1;
    for (int q = threadIdx.x; q < sp.z; q += blockDim.x) {
        const int64_t pos = (int64_t)sp.y + q;
        const int32_t src = perm[pos];
        const T a = alpha_double ? (T)(static_cast<const double*>(alpha)[src])
                                 : (T)(static_cast<const float*>(alpha)[src]);
        T w[DA][2 * kMaxM + 1];
        int off[DA];
        node_weights<T, DA>(cell, frac, N, pos, bc, Tb, m, b, norm, tap, w, off);
        if (DA == 1) {
            for (int k0 = 0; k0 < ntap; k0++) atomicAdd(&acc[off[0] + k0], a * w[0][k0]);
        } else if (DA == 2) {
            for (int k0 = 0; k0 < ntap; k0++) {
                const T a0 = a * w[0][k0];
                T* row = acc + (off[0] + k0) * R + off[DA - 1];
                for (int k1 = 0; k1 < ntap; k1++) atomicAdd(row + k1, a0 * w[DA - 1][k1]);
            }
        } else {
            for (int k0 = 0; k0 < ntap; k0++) {
                const T a0 = a * w[0][k0];
                for (int k1 = 0; k1 < ntap; k1++) {
                    const T a01 = a0 * w[1 % DA][k1];
                    T* row = acc + ((off[0] + k0) * R + off[1 % DA] + k1) * R + off[DA - 1];
                    for (int k2 = 0; k2 < ntap; k2++) atomicAdd(row + k2, a01 * w[DA - 1][k2]);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RD; i += blockDim.x) {
        const T v = acc[i];
        if (v != T(0)) atomicAdd(&grid[region_to_grid<T, DA>(i, R, bc, Tb, m, nos)], v);
    }
}

template <typename T, int DA>
__global__ void __launch_bounds__(kThreads)
k_gather(const int4* __restrict__ sub, const int32_t* __restrict__ perm, const int32_t* __restrict__ cell,
         const T* __restrict__ frac, int64_t N, const T* __restrict__ h, int nos, int Tb, int nb, int R,
         int m, T b, T norm, T* __restrict__ out, const double* __restrict__ tap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* reg = reinterpret_cast<T*>(smem_raw);
    const int4 sp = sub[blockIdx.x];
    int bc[3] = {0, 0, 0};
    bin_coords<T, DA>(sp.x, nb, bc);
    int RD = R;
    if (DA > 1) RD *= R;
    if (DA > 2) RD *= R;
    for (int i = threadIdx.x; i < RD; i += blockDim.x) reg[i] = h[region_to_grid<T, DA>(i, R, bc, Tb, m, nos)];
    __syncthreads();
    const int ntap = 2 * m + 1;
    for (int q = threadIdx.x; q < sp.z; q += blockDim.x) {
        const int64_t pos = (int64_t)sp.y + q;
        T w[DA][2 * kMaxM + 1];
        int off[DA];
        node_weights<T, DA>(cell, frac, N, pos, bc, Tb, m, b, norm, tap, w, off);
        T acc = T(0);
        if (DA == 1) {
            for (int k0 = 0; k0 < ntap; k0++) acc += reg[off[0] + k0] * w[0][k0];
        } else if (DA == 2) {
            for (int k0 = 0; k0 < ntap; k0++) {
                const T* row = reg + (off[0] + k0) * R + off[DA - 1];
                T s = T(0);
                for (int k1 = 0; k1 < ntap; k1++) s += row[k1] * w[DA - 1][k1];
                acc += w[0][k0] * s;
            }
        } else {
            for (int k0 = 0; k0 < ntap; k0++) {
                T s0 = T(0);
                for (int k1 = 0; k1 < ntap; k1++) {
                    const T* row = reg + ((off[0] + k0) * R + off[1 % DA] + k1) * R + off[DA - 1];
                    T s = T(0);
                    for (int k2 = 0; k2 < ntap; k2++) s += row[k2] * w[DA - 1][k2];
                    s0 += w[1 % DA][k1] * s;
                }
                acc += w[0][k0] * s0;
            }
        }
        out[perm[pos]] = acc;
    }
}

static int region_elems(const WindowPlan& w) {
    int r = 1;
    for (int t = 0; t < w.dA; t++) r *= w.R;
    return r;
}

template <typename K>
static void allow_big_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T>
static const T* frac_of(const PointSet& ps);
template <>
const double* frac_of<double>(const PointSet& ps) { return ps.frac64; }
template <>
const float* frac_of<float>(const PointSet& ps) { return ps.frac32; }

template <typename T>
anova_status spread_window(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const void* alpha,
                           int alpha_is_double, T* grid, cudaStream_t st) {
    if (ps.nsub == 0) return ANOVA_OK;
    if (w.dense && w.dA == 3) return spread3_dense<T>(plan, w, ps, alpha, alpha_is_double, grid, st);
    const size_t sh = (size_t)region_elems(w) * sizeof(T);
    const T b = (T)plan->b, norm = (T)plan->psi_norm;
    const T* frac = frac_of<T>(ps);
    // the FP64 tap table describes the plan's own nodes
    const double* tap = (sizeof(T) == 8 && &ps == &w.X) ? w.wtap64 : nullptr;
#define ANOVA_SPREAD(DA_)                                                                    \
    {                                                                                        \
        auto k = k_spread<T, DA_>;                                                           \
        static bool once = (allow_big_smem(k), true);                                        \
        (void)once;                                                                          \
        k<<<ps.nsub, kThreads, sh, st>>>(ps.sub, ps.perm, ps.cell, frac, ps.N, alpha,          \
                                         alpha_is_double, grid, w.nos, w.T, w.nb, w.R, plan->m, b, norm, tap); \
    }
    if (w.dA == 1) ANOVA_SPREAD(1) else if (w.dA == 2) ANOVA_SPREAD(2) else ANOVA_SPREAD(3)
#undef ANOVA_SPREAD
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template <typename T>
anova_status gather_window(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const T* h, T* out,
                           cudaStream_t st) {
    if (ps.nsub == 0) return ANOVA_OK;
    if (w.dense && w.dA == 3) return gather3_dense<T>(plan, w, ps, h, out, st);
    const size_t sh = (size_t)region_elems(w) * sizeof(T);
    const T b = (T)plan->b, norm = (T)plan->psi_norm;
    const T* frac = frac_of<T>(ps);
    const double* tap = (sizeof(T) == 8 && &ps == &w.X) ? w.wtap64 : nullptr;
#define ANOVA_GATHER(DA_)                                                                    \
    {                                                                                        \
        auto k = k_gather<T, DA_>;                                                           \
        static bool once = (allow_big_smem(k), true);                                        \
        (void)once;                                                                          \
        k<<<ps.nsub, kThreads, sh, st>>>(ps.sub, ps.perm, ps.cell, frac, ps.N, h, w.nos, w.T,  \
                                         w.nb, w.R, plan->m, b, norm, out, tap);             \
    }
    if (w.dA == 1) ANOVA_GATHER(1) else if (w.dA == 2) ANOVA_GATHER(2) else ANOVA_GATHER(3)
#undef ANOVA_GATHER
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template anova_status spread_window<double>(anova_plan*, const WindowPlan&, const PointSet&, const void*,
                                            int, double*, cudaStream_t);
template anova_status spread_window<float>(anova_plan*, const WindowPlan&, const PointSet&, const void*,
                                           int, float*, cudaStream_t);
template anova_status gather_window<double>(anova_plan*, const WindowPlan&, const PointSet&, const double*,
                                            double*, cudaStream_t);
template anova_status gather_window<float>(anova_plan*, const WindowPlan&, const PointSet&, const float*,
                                           float*, cudaStream_t);

}  // namespace anova
