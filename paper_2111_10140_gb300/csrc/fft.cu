// fft.cu -- the FFT / multiply / inverse-FFT middle of the fast summation
// (arXiv 2111.10140, Sec. 4.2 Eq. fastsum, Sec. 4.3 K ~= Phi D Phi^*):
//
//   G_k = sum_{u in I_nos} g_u e^{-2 pi i k.u / nos},  k in I_n   (pruned forward)
//   H_k = D_k G_k
//   h_u = Re sum_{k in I_n} H_k e^{+2 pi i k.u / nos}             (zero-padded inverse)
//
// done one axis at a time, each pass a pruned DFT along that axis: forward
// from the last axis to the first (the first pass reads the real grid, the
// last multiplies by D), inverse from the first axis to the last (the last
// pass writes only the real part into the grid).
#include <cuda_runtime.h>

#include "common.cuh"

namespace anova {

template <typename T>
struct Cplx;
template <>
struct Cplx<double> { using type = double2; };
template <>
struct Cplx<float> { using type = float2; };

// out[(o0, o, s)] = sum_i in[(o0, i, s)] * w(k u),  u = i - Lin/2, k = o - Lout/2,
// w(r) = tw[r mod nos] (forward, e^{-2 pi i r/nos}) or its conjugate (inverse).
template <typename T, bool IN_REAL, bool OUT_REAL>
__global__ void __launch_bounds__(kThreads)
k_dft_axis(const void* __restrict__ in_, void* __restrict__ out_, int64_t outer, int Lin, int64_t inner,
           int Lout, int nos, const typename Cplx<T>::type* __restrict__ tw, int inverse,
           const T* __restrict__ D) {
    using C = typename Cplx<T>::type;
    const int64_t tot = outer * Lout * inner;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx % inner;
        const int o = (int)((idx / inner) % Lout);
        const int64_t o0 = idx / (inner * Lout);
        const int k = o - Lout / 2;
        T ar = T(0), ai = T(0);
        int r = (int)(((int64_t)k * (-Lin / 2)) % nos);
        if (r < 0) r += nos;
        int kstep = k % nos;
        if (kstep < 0) kstep += nos;
        const int64_t base = o0 * Lin * inner + s;
        for (int i = 0; i < Lin; i++) {
            C w = tw[r];
            if (inverse) w.y = -w.y;
            if (IN_REAL) {
                const T x = static_cast<const T*>(in_)[base + (int64_t)i * inner];
                ar += x * w.x;
                ai += x * w.y;
            } else {
                const C x = static_cast<const C*>(in_)[base + (int64_t)i * inner];
                ar += x.x * w.x - x.y * w.y;
                ai += x.x * w.y + x.y * w.x;
            }
            r += kstep;
            if (r >= nos) r -= nos;
        }
        if (D) {
            const T dk = D[idx];
            ar *= dk;
            ai *= dk;
        }
        if (OUT_REAL) {
            static_cast<T*>(out_)[idx] = ar;
        } else {
            C v;
            v.x = ar;
            v.y = ai;
            static_cast<C*>(out_)[idx] = v;
        }
    }
}

template <typename T>
static const typename Cplx<T>::type* tw_of(const WindowPlan& w);
template <>
const double2* tw_of<double>(const WindowPlan& w) { return w.tw64; }
template <>
const float2* tw_of<float>(const WindowPlan& w) { return w.tw32; }
template <typename T>
static const T* D_of(const WindowPlan& w);
template <>
const double* D_of<double>(const WindowPlan& w) { return w.D64; }
template <>
const float* D_of<float>(const WindowPlan& w) { return w.D32; }

// In place on `grid` (real, nos^dA): grid <- Re IDFT(D . DFT(grid)).
template <typename T>
anova_status fft_convolve_window(anova_plan* plan, const WindowPlan& w, T* grid, cudaStream_t st) {
    const int dA = w.dA, n = w.n, nos = w.nos;
    const auto* tw = tw_of<T>(w);
    const T* D = D_of<T>(w);
    using C = typename Cplx<T>::type;
    void* bufs[2] = {static_cast<C*>(plan->work1) + w.work_off, static_cast<C*>(plan->work2) + w.work_off};
    int cur = 0;
    const int cap = 8 * plan->sm_count;
    // extents per axis: axes < t already transformed (n), axes >= t not yet (nos)
    auto launch = [&](auto kern, const void* in, void* out, int64_t outer, int Lin, int64_t inner, int Lout,
                      int inverse, const T* Dm) {
        int64_t tot = outer * Lout * inner;
        kern<<<grid_for(tot, kThreads, cap), kThreads, 0, st>>>(in, out, outer, Lin, inner, Lout, nos, tw,
                                                                inverse, Dm);
    };
    // forward, last axis first
    const void* src = grid;
    for (int t = dA - 1; t >= 0; t--) {
        int64_t outer = 1, inner = 1;
        for (int i = 0; i < t; i++) outer *= nos;
        for (int i = t + 1; i < dA; i++) inner *= n;
        void* dst = bufs[cur];
        const T* Dm = (t == 0) ? D : nullptr;
        if (t == dA - 1)
            launch(k_dft_axis<T, true, false>, src, dst, outer, nos, inner, n, 0, Dm);
        else
            launch(k_dft_axis<T, false, false>, src, dst, outer, nos, inner, n, 0, Dm);
        src = dst;
        cur ^= 1;
    }
    // inverse, first axis first
    for (int t = 0; t < dA; t++) {
        int64_t outer = 1, inner = 1;
        for (int i = 0; i < t; i++) outer *= nos;
        for (int i = t + 1; i < dA; i++) inner *= n;
        if (t == dA - 1) {
            launch(k_dft_axis<T, false, true>, src, grid, outer, n, inner, nos, 1, nullptr);
        } else {
            void* dst = bufs[cur];
            launch(k_dft_axis<T, false, false>, src, dst, outer, n, inner, nos, 1, nullptr);
            src = dst;
            cur ^= 1;
        }
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template anova_status fft_convolve_window<double>(anova_plan*, const WindowPlan&, double*, cudaStream_t);
template anova_status fft_convolve_window<float>(anova_plan*, const WindowPlan&, float*, cudaStream_t);

}  // namespace anova
