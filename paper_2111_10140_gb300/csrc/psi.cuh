// psi.cuh -- the normalised Kaiser-Bessel window of the FP32 kernels, evaluated
// on the fly from a node's cell and offset (the window of the NFFT, Sec. 4.1,
// with the parameters of the Kaiser-Bessel choice): per unit interval q the
// plan fits psi(q - m + f), f in [0, 1), with a polynomial in (f - 1/2) in
// FP64 and keeps it in FP32; the coefficients travel as a kernel parameter, so
// the evaluation reads them from the constant bank at compile-time offsets.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "common.cuh"

namespace anova {

template <int M>
struct PsiCoef {
    float c[2 * M][kPsiStride];     // interval q: psi(q - M + f) ~ sum_k c[q][k] (f - 1/2)^k
};

// psi(q - M + f) for q in [0, 2M); the coefficients are compile-time offsets into the parameter bank
template <int M>
__device__ __forceinline__ void psi_taps(const PsiCoef<M>& P, float f, float (&t)[2 * M]) {
    const float u = f - 0.5f;
#pragma unroll
    for (int q = 0; q < 2 * M; q++) {
        float acc = P.c[q][kPsiDeg];
#pragma unroll
        for (int k = kPsiDeg - 1; k >= 0; k--) acc = fmaf(acc, u, P.c[q][k]);
        t[q] = acc;
    }
}

// region row r of a node in cell c of its bin: psi(c + M - r + f) = t[c + 2M - r]
// where that tap exists, 0 elsewhere (and for r >= R)
template <int R, int M>
__device__ __forceinline__ void place_taps(const float (&t)[2 * M], int c, float (&w)[16]) {
    constexpr int TB = R - 2 * M;
#pragma unroll
    for (int r = 0; r < 16; r++) {
        float v = 0.f;
#pragma unroll
        for (int cc = 0; cc < TB; cc++) {
            const int q = cc + 2 * M - r;
            if (q >= 0 && q < 2 * M) v = (c == cc) ? t[q] : v;
        }
        w[r] = v;
    }
}

__device__ __forceinline__ int wrap_cell(int g, int nos) { return g < 0 ? g + nos : (g >= nos ? g - nos : g); }

// the kernel parameter for cutoff M from the plan's host copy of the coefficients
template <int M>
inline PsiCoef<M> psi_coef(const float* psi_host) {
    PsiCoef<M> P;
    std::memcpy(P.c, psi_host, sizeof(P.c));
    return P;
}

}  // namespace anova
