// direct.cu -- the direct ANOVA-Gaussian kernel sum on the GPU (arXiv 2111.10140,
// Sec. 2 Eq. mult_with_K and Sec. 4.2 Eq. kernelsum with the kernel of Sec. 3
// Eq. extended_Gaussian_ANOVA_kernel):
//
//   out_i = sum_l eta_l sum_j alpha_j exp(-||z_i^{W_l} - x_j^{W_l}||^2 / ell^2)
//
// O(M N P) work, no approximation: the reference for the fast summation's
// accuracy and the "dense" side of the direct-versus-fast comparison.  One
// thread per output row; the nodes x_j stream through shared memory in tiles.
// FP64: everything in double.  FP32: coordinates, exponentials and the sums
// over one tile in float (exp via the fast hardware exponential), tile sums
// accumulated in double.  The window table travels as a kernel argument.
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace anova {

constexpr int kDirectTile = 256;

struct DirectWindows {
    int P;
    int dA[kMaxWindows];
    int feat[kMaxWindows][3];
    double eta[kMaxWindows];
};

template <typename T>
__device__ __forceinline__ T dexp(T x);
template <>
__device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float dexp<float>(float x) { return __expf(x); }

template <typename T>
__global__ void __launch_bounds__(kDirectTile)
k_direct(const double* __restrict__ Z, int64_t M, int64_t ldz, const double* __restrict__ X, int64_t N,
         int64_t ldx, const DirectWindows wins, double inv_ell2, const double* __restrict__ alpha,
         double* __restrict__ out) {
    __shared__ T sx[kDirectTile][3];
    __shared__ T sa[kDirectTile];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = i < M;
    const int P = wins.P;
    const T ie = (T)inv_ell2;
    double total = 0.0;
    for (int l = 0; l < P; l++) {
        const int dA = wins.dA[l];
        const int f0 = wins.feat[l][0], f1 = wins.feat[l][1], f2 = wins.feat[l][2];
        T z0 = 0, z1 = 0, z2 = 0;
        if (valid) {
            z0 = (T)Z[i * ldz + f0];
            if (dA > 1) z1 = (T)Z[i * ldz + f1];
            if (dA > 2) z2 = (T)Z[i * ldz + f2];
        }
        double sl = 0.0;
        for (int64_t j0 = 0; j0 < N; j0 += kDirectTile) {
            const int cnt = (int)((N - j0 < kDirectTile) ? (N - j0) : kDirectTile);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int64_t j = j0 + threadIdx.x;
                sx[threadIdx.x][0] = (T)X[j * ldx + f0];
                sx[threadIdx.x][1] = (dA > 1) ? (T)X[j * ldx + f1] : T(0);
                sx[threadIdx.x][2] = (dA > 2) ? (T)X[j * ldx + f2] : T(0);
                sa[threadIdx.x] = (T)alpha[j];
            }
            __syncthreads();
            T acc = T(0);
            for (int k = 0; k < cnt; k++) {
                const T d0 = z0 - sx[k][0], d1 = z1 - sx[k][1], d2 = z2 - sx[k][2];
                const T r2 = d0 * d0 + d1 * d1 + d2 * d2;
                acc += sa[k] * dexp<T>(-r2 * ie);
            }
            sl += (double)acc;
        }
        total += wins.eta[l] * sl;
    }
    if (valid) out[i] = total;
}

}  // namespace anova

using namespace anova;

extern "C" anova_status anova_direct_matvec(const double* Z, int64_t M, int64_t ldz, const double* X, int64_t N,
                                            int64_t ldx, int32_t d, const int32_t* windows, int32_t P,
                                            const double* weights, double ell, int32_t dtype, const double* alpha,
                                            double* out, void* stream) {
    if (M < 0 || N < 0 || d < 1 || ldz < d || ldx < d || !windows || P < 1 || P > kMaxWindows ||
        !(ell > 0.0) || (dtype != ANOVA_FP64 && dtype != ANOVA_FP32) || (M > 0 && (!Z || !out)) ||
        (N > 0 && (!X || !alpha))) {
        set_error("anova_direct_matvec: bad sizes, windows, ell, dtype or pointers");
        return ANOVA_EINVAL;
    }
    DirectWindows hw;
    hw.P = P;
    for (int l = 0; l < P; l++) {
        int dA = 0;
        while (dA < 3 && windows[3 * l + dA] >= 0) dA++;
        if (dA == 0) {
            set_error("anova_direct_matvec: empty window");
            return ANOVA_EINVAL;
        }
        for (int t = 0; t < 3; t++) {
            const int f = (t < dA) ? windows[3 * l + t] : windows[3 * l];
            if (f < 0 || f >= d) {
                set_error("anova_direct_matvec: feature index out of range");
                return ANOVA_EINVAL;
            }
            hw.feat[l][t] = f;
        }
        hw.dA[l] = dA;
        hw.eta[l] = weights ? weights[l] : 1.0 / P;
    }
    if (M == 0) return ANOVA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)((M + kDirectTile - 1) / kDirectTile);
    const double inv_ell2 = 1.0 / (ell * ell);
    if (dtype == ANOVA_FP64)
        k_direct<double><<<blocks, kDirectTile, 0, st>>>(Z, M, ldz, X, N, ldx, hw, inv_ell2, alpha, out);
    else
        k_direct<float><<<blocks, kDirectTile, 0, st>>>(Z, M, ldz, X, N, ldx, hw, inv_ell2, alpha, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("anova_direct_matvec: ") + cudaGetErrorString(e));
        return ANOVA_ECUDA;
    }
    return ANOVA_OK;
}
