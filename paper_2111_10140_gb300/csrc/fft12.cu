// fft12.cu -- the FFT / multiply / inverse-FFT middle of the fast summation
// (arXiv 2111.10140, Sec. 4.2 Eq. fastsum) for every 1-D and 2-D window of a
// plan in one launch: one thread block per window, the whole transform in
// shared memory.
//
// Only the box of grid cells that the window's nodes touch (their cell range
// plus the window's cut-off, per axis) is non-zero after the spread, and the
// gather on the same nodes reads only that box.  So the forward DFT sums over
// the box and the inverse DFT is evaluated on the box only:
//
//   A[j0][k1] = sum_{j1 in box} g[j0][j1] w(k1 u1(j1))          (axis 1)
//   H[k0][k1] = D[k0][k1] sum_{j0 in box} A[j0][k1] w(k0 u0(j0))  (axis 0, times D)
//   C[j0][k1] = sum_{k0} H[k0][k1] conj w(k0 u0(j0))             (inverse axis 0)
//   h[j0][j1] = Re sum_{k1} C[j0][k1] conj w(k1 u1(j1))          (inverse axis 1)
//
// with k in I_n (centred), u the centred grid index of a box cell and
// w(r) = e^{-2 pi i r / nos}.  A 1-D window is the same with one box row and
// no axis-0 passes.  Cells outside the box keep stale values; nothing reads
// them in a matrix-vector product.
#include <cuda_runtime.h>

#include "common.cuh"

namespace anova {

template <typename T>
struct Cplx12;
template <>
struct Cplx12<double> { using type = double2; };
template <>
struct Cplx12<float> { using type = float2; };

constexpr int kFft12Threads = 1024;

__host__ __device__ inline size_t fft12_smem(int dA, int n, int nos, int B0, int B1, size_t real_bytes) {
    const size_t c = 2 * real_bytes;
    const int n0 = dA == 2 ? n : 1;
    size_t b = (size_t)nos * c + (size_t)B0 * n * c + (size_t)n0 * n * c + (size_t)B0 * B1 * real_bytes;
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ int mod_pos(int64_t a, int m) {
    int r = (int)(a % m);
    return r < 0 ? r + m : r;
}

// NC > 0: every window of the launch has n = NC and n_os = 2 NC
template <typename T, int NC = 0>
__global__ void __launch_bounds__(kFft12Threads)
k_fft12_box(const Fft12Win* __restrict__ descs) {
    using C = typename Cplx12<T>::type;
    const Fft12Win d = descs[blockIdx.x];
    if (d.live && !*d.live) return;   // a batch system that has stopped
    const int n = NC ? NC : d.n, nos = NC ? 2 * NC : d.nos, half = nos / 2;
    const bool two = d.dA == 2;
    const int B0 = two ? d.B[0] : 1, B1 = two ? d.B[1] : d.B[0];
    const int lo0 = two ? d.lo[0] : 0, lo1 = two ? d.lo[1] : d.lo[0];
    const int n0 = two ? n : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    C* s_tw = reinterpret_cast<C*>(smem);
    C* s_A = s_tw + nos;
    C* s_H = s_A + (size_t)B0 * n;
    T* s_g = reinterpret_cast<T*>(s_H + (size_t)n0 * n);
    T* grid = static_cast<T*>(d.grid);
    const C* tw = static_cast<const C*>(d.tw);
    const T* D = static_cast<const T*>(d.D);
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int i = tid; i < nos; i += nt) s_tw[i] = tw[i];
    // box cells (i0, i1) = ((lo0 + j0) mod nos, (lo1 + j1) mod nos)
    for (int idx = tid; idx < B0 * B1; idx += nt) {
        const int j0 = idx / B1, j1 = idx - j0 * B1;
        const int i0 = two ? mod_pos(lo0 + j0, nos) : 0;
        const int i1 = mod_pos(lo1 + j1, nos);
        s_g[idx] = grid[(size_t)i0 * nos + i1];
    }
    __syncthreads();
    // u of the first box cell per axis; u advances by 1 per box cell (a wrap
    // changes u by nos, which leaves every k u mod nos unchanged)
    const int u0s = (two ? mod_pos(lo0, nos) : half) - half;
    const int u1s = mod_pos(lo1, nos) - half;

    // forward along axis 1: A[j0][k1]
    for (int idx = tid; idx < B0 * n; idx += nt) {
        const int j0 = idx / n, o1 = idx - j0 * n;
        const int k1 = o1 - n / 2;
        int r = mod_pos((int64_t)k1 * u1s, nos);
        const int step = mod_pos(k1, nos);
        const T* row = s_g + (size_t)j0 * B1;
        T ar = T(0), ai = T(0);
        for (int j1 = 0; j1 < B1; j1++) {
            const C w = s_tw[r];
            const T x = row[j1];
            ar += x * w.x;
            ai += x * w.y;
            r += step;
            if (r >= nos) r -= nos;
        }
        C v;
        v.x = ar;
        v.y = ai;
        s_A[idx] = v;
    }
    __syncthreads();
    // forward along axis 0 and the multiplier: H[k0][k1]
    for (int idx = tid; idx < n0 * n; idx += nt) {
        const T dk = D[idx];
        C v;
        if (two) {
            const int o0 = idx / n, o1 = idx - o0 * n;
            const int k0 = o0 - n / 2;
            int r = mod_pos((int64_t)k0 * u0s, nos);
            const int step = mod_pos(k0, nos);
            T ar = T(0), ai = T(0);
            for (int j0 = 0; j0 < B0; j0++) {
                const C w = s_tw[r];
                const C x = s_A[(size_t)j0 * n + o1];
                ar += x.x * w.x - x.y * w.y;
                ai += x.x * w.y + x.y * w.x;
                r += step;
                if (r >= nos) r -= nos;
            }
            v.x = ar * dk;
            v.y = ai * dk;
        } else {
            const C x = s_A[idx];
            v.x = x.x * dk;
            v.y = x.y * dk;
        }
        s_H[idx] = v;
    }
    __syncthreads();
    // inverse along axis 0 on the box rows: C[j0][k1] (into s_A)
    const C* s_C = s_H;
    if (two) {
        for (int idx = tid; idx < B0 * n; idx += nt) {
            const int j0 = idx / n, o1 = idx - j0 * n;
            const int u0 = u0s + j0;
            int r = mod_pos((int64_t)(-n / 2) * u0, nos);   // k0 = -n/2 first
            const int step = mod_pos(u0, nos);               // k0 advances by 1
            T ar = T(0), ai = T(0);
            for (int o0 = 0; o0 < n; o0++) {
                const C w = s_tw[r];
                const C x = s_H[(size_t)o0 * n + o1];
                ar += x.x * w.x + x.y * w.y;    // x * conj(w)
                ai += x.y * w.x - x.x * w.y;
                r += step;
                if (r >= nos) r -= nos;
            }
            C v;
            v.x = ar;
            v.y = ai;
            s_A[idx] = v;
        }
        __syncthreads();
        s_C = s_A;
    }
    // inverse along axis 1 on the box cells, real part, back into the grid
    for (int idx = tid; idx < B0 * B1; idx += nt) {
        const int j0 = idx / B1, j1 = idx - j0 * B1;
        const int u1 = u1s + j1;
        int r = mod_pos((int64_t)(-n / 2) * u1, nos);
        const int step = mod_pos(u1, nos);
        const C* row = s_C + (size_t)j0 * n;
        T acc = T(0);
        for (int o1 = 0; o1 < n; o1++) {
            const C w = s_tw[r];
            const C x = row[o1];
            acc += x.x * w.x + x.y * w.y;
            r += step;
            if (r >= nos) r -= nos;
        }
        const int i0 = two ? mod_pos(lo0 + j0, nos) : 0;
        const int i1 = mod_pos(lo1 + j1, nos);
        grid[(size_t)i0 * nos + i1] = acc;
    }
}

bool fft12_box_supported(const WindowPlan& w) {
    if (w.dA < 1 || w.dA > 2) return false;
    const int B0 = w.dA == 2 ? w.box_ext[0] : 1, B1 = w.dA == 2 ? w.box_ext[1] : w.box_ext[0];
    return fft12_smem(w.dA, w.n, w.nos, B0, B1, sizeof(double)) <= kFft12MaxSmem;
}

size_t fft12_window_smem(const WindowPlan& w, size_t real_bytes) {
    const int B0 = w.dA == 2 ? w.box_ext[0] : 1, B1 = w.dA == 2 ? w.box_ext[1] : w.box_ext[0];
    return fft12_smem(w.dA, w.n, w.nos, B0, B1, real_bytes);
}

template <typename T, int NC>
static void launch_fft12(const Fft12Win* desc, int nw, size_t smem, cudaStream_t st) {
    static bool attrs = [] {
        cudaFuncSetAttribute(k_fft12_box<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFft12MaxSmem);
        return true;
    }();
    (void)attrs;
    k_fft12_box<T, NC><<<nw, kFft12Threads, smem, st>>>(desc);
}

template <typename T>
anova_status fft12_box_run(const Fft12Win* desc, int nw, size_t smem, cudaStream_t st, int uniform_n) {
    if (nw == 0) return ANOVA_OK;
    switch (uniform_n) {
        case 16: launch_fft12<T, 16>(desc, nw, smem, st); break;
        case 32: launch_fft12<T, 32>(desc, nw, smem, st); break;
        case 64: launch_fft12<T, 64>(desc, nw, smem, st); break;
        default: launch_fft12<T, 0>(desc, nw, smem, st); break;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template <typename T>
anova_status fft12_box_all(anova_plan* plan, cudaStream_t st) {
    const int nw = (int)plan->fft12_windows.size();
    const size_t sh = sizeof(T) == 8 ? plan->fft12_smem64 : plan->fft12_smem32;
    return fft12_box_run<T>(plan->fft12_desc + (sizeof(T) == 8 ? 0 : nw), nw, sh, st, plan->fft12_uniform_n);
}

template anova_status fft12_box_run<double>(const Fft12Win*, int, size_t, cudaStream_t, int);
template anova_status fft12_box_run<float>(const Fft12Win*, int, size_t, cudaStream_t, int);
template anova_status fft12_box_all<double>(anova_plan*, cudaStream_t);
template anova_status fft12_box_all<float>(anova_plan*, cudaStream_t);

}  // namespace anova
