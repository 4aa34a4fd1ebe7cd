// fft3.cu -- the FFT / multiply / inverse-FFT middle of the fast summation
// for 3-D windows, restricted to the box of grid cells the nodes touch and
// batched over windows (arXiv 2111.10140, Sec. 4.2 Eq. fastsum, Sec. 4.3):
//
//   G_k = sum_{u in box} g_u e^{-2 pi i k.u/nos},  k in I_n^3
//   h_u = Re sum_{k in I_n^3} D_k G_k e^{+2 pi i k.u/nos},  u in box
//
// Spreading writes only inside the box and gathering reads only inside it,
// so every other grid cell contributes nothing and is never needed.  The box
// is the union of the regions of the occupied bins (or the whole torus when
// that union would wrap onto itself).  Passes, with box extents Bx, By, Bz:
//   F1  z -> kz:   (Bx, By, Bz) real      -> (Bx, By, n)  complex
//   F2  y -> ky:   (Bx, By, n)            -> (Bx, n, n)
//   M   x -> kx, multiply by D, kx -> x:  (Bx, n, n) -> (Bx, n, n)
//   I2  ky -> y:   (Bx, n, n)             -> (Bx, By, n)
//   I3  kz -> z:   (Bx, By, n)            -> (Bx, By, Bz), real part into the grid
//
// Twiddles: consecutive box cells have consecutive values modulo nos, so the
// table index (k u mod nos) advances by a constant step along every loop.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace anova {

template <typename T>
struct C2;
template <>
struct C2<double> { using type = double2; };
template <>
struct C2<float> { using type = float2; };

__device__ __forceinline__ int modp(int v, int p) {
    v %= p;
    return v < 0 ? v + p : v;
}

// centred value of box coordinate 0 on an axis starting at grid index lo
__device__ __forceinline__ int box_value0(int lo, int nos) { return modp(lo, nos) - nos / 2; }

// acc += v * w (complex), with conj(w) when inverse
template <typename C, typename T>
__device__ __forceinline__ void cmac(const C& v, C w, int inverse, T& ar, T& ai) {
    if (inverse) w.y = -w.y;
    ar = fma(v.x, w.x, fma(-v.y, w.y, ar));
    ai = fma(v.x, w.y, fma(v.y, w.x, ai));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft3_f1(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const T* __restrict__ g = static_cast<const T*>(W.grid);
    C* __restrict__ A = static_cast<C*>(W.buf1);
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    const int n = W.n, nos = W.nos;
    const int64_t tot = (int64_t)W.B[0] * W.B[1] * n;
    const int z0v = box_value0(W.lo[2], nos);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % n) - n / 2;
        const int y = (int)((idx / n) % W.B[1]);
        const int x = (int)(idx / ((int64_t)n * W.B[1]));
        const int64_t row = ((int64_t)modp(W.lo[0] + x, nos) * nos + modp(W.lo[1] + y, nos)) * nos;
        int r = modp(kz * z0v, nos);
        const int step = modp(kz, nos);
        int gz = modp(W.lo[2], nos);
        T ar = T(0), ai = T(0);
        for (int z = 0; z < W.B[2]; z++) {
            const T v = g[row + gz];
            const C w = tw[r];
            ar = fma(v, w.x, ar);
            ai = fma(v, w.y, ai);
            r += step;
            if (r >= nos) r -= nos;
            if (++gz == nos) gz = 0;
        }
        C o;
        o.x = ar;
        o.y = ai;
        A[idx] = o;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft3_f2(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const C* __restrict__ A = static_cast<const C*>(W.buf1);
    C* __restrict__ Bo = static_cast<C*>(W.buf2);
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    const int n = W.n, nos = W.nos, By = W.B[1];
    const int64_t tot = (int64_t)W.B[0] * n * n;
    const int y0v = box_value0(W.lo[1], nos);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % n);
        const int ky = (int)((idx / n) % n) - n / 2;
        const int x = (int)(idx / ((int64_t)n * n));
        int r = modp(ky * y0v, nos);
        const int step = modp(ky, nos);
        T ar = T(0), ai = T(0);
        const C* a = A + (int64_t)x * By * n + kz;
#pragma unroll 4
        for (int y = 0; y < By; y++) {
            cmac(a[(int64_t)y * n], tw[r], 0, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        C o;
        o.x = ar;
        o.y = ai;
        Bo[idx] = o;
    }
}

// Fused middle pass along x for up to 32 consecutive kz of one ky per block:
// H[kx] = D[kx] sum_x B[x] e^{-2 pi i kx x/nos}, then C[x] = sum_kx H[kx] e^{+...}.
constexpr int kMidLanes = 32, kMidWarps = 32, kMaxN3 = 64, kMaxBox3 = 256;
constexpr int kSlabParts = 1;   // blocks per slab in the slab kernels (kz columns forward, y rows inverse);
                                // 2 and 4 measured slower on the mid workload (duplicated staging)
// Dynamic shared memory: H (n x 32), the staged lines (Bx x 32) when Bx <= kMidStage, twiddles (nos).
constexpr int kMidStage = 64;
// NC > 0: every window of the launch has n = NC and n_os = 2 NC (index arithmetic on constants)
template <typename T, int NC = 0>
__global__ void __launch_bounds__(kMidLanes * kMidWarps) k_fft3_mid(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char mid_raw[];
    C (*sH)[kMidLanes] = reinterpret_cast<C (*)[kMidLanes]>(mid_raw);
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const int n = NC ? NC : W.n, nos = NC ? 2 * NC : W.nos, Bx = W.B[0];
    const int lines_per_ky = (n + kMidLanes - 1) / kMidLanes;
    if ((int)blockIdx.x >= n * lines_per_ky) return;
    const int lane = threadIdx.x % kMidLanes, warp = threadIdx.x / kMidLanes;
    const int ky = blockIdx.x / lines_per_ky;
    const int kz = (blockIdx.x % lines_per_ky) * kMidLanes + lane;
    const bool ok = kz < n;
    const C* __restrict__ Bi = static_cast<const C*>(W.buf2);
    C* __restrict__ Co = static_cast<C*>(W.buf1);
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    const T* __restrict__ D = static_cast<const T*>(W.D);
    const int x0v = box_value0(W.lo[0], nos);
    const bool staged = Bx <= kMidStage;
    C (*sBx)[kMidLanes] = sH + kMaxN3;              // the block's 32 lines, x < Bx
    C* stw = reinterpret_cast<C*>(sBx + kMidStage); // twiddles
    for (int i = threadIdx.x; i < nos; i += blockDim.x) stw[i] = tw[i];
    if (staged)
        for (int x = warp; x < Bx; x += kMidWarps) {
            C v;
            v.x = T(0);
            v.y = T(0);
            if (ok) v = Bi[((int64_t)x * n + ky) * n + kz];
            sBx[x][lane] = v;
        }
    __syncthreads();
    for (int kx = warp; kx < n; kx += kMidWarps) {
        const int kxv = kx - n / 2;
        int r = modp(kxv * x0v, nos);
        const int step = modp(kxv, nos);
        T ar = T(0), ai = T(0);
#pragma unroll 4
        for (int x = 0; x < Bx; x++) {
            C v;
            if (staged) {
                v = sBx[x][lane];
            } else {
                v.x = T(0);
                v.y = T(0);
                if (ok) v = Bi[((int64_t)x * n + ky) * n + kz];
            }
            cmac(v, stw[r], 0, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        const T dk = ok ? D[((int64_t)kx * n + ky) * n + kz] : T(0);
        C h;
        h.x = ar * dk;
        h.y = ai * dk;
        sH[kx][lane] = h;
    }
    __syncthreads();
    for (int x = warp; x < Bx; x += kMidWarps) {
        const int xv = modp(W.lo[0] + x, nos) - nos / 2;
        int r = modp((-n / 2) * xv, nos);
        const int step = modp(xv, nos);
        T ar = T(0), ai = T(0);
#pragma unroll 4
        for (int kx = 0; kx < n; kx++) {
            cmac(sH[kx][lane], stw[r], 1, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        if (ok) {
            C o;
            o.x = ar;
            o.y = ai;
            Co[((int64_t)x * n + ky) * n + kz] = o;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft3_i2(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const C* __restrict__ Ci = static_cast<const C*>(W.buf1);
    C* __restrict__ E = static_cast<C*>(W.buf2);
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    const int n = W.n, nos = W.nos, By = W.B[1];
    const int64_t tot = (int64_t)W.B[0] * By * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(idx % n);
        const int y = (int)((idx / n) % By);
        const int x = (int)(idx / ((int64_t)n * By));
        const int yv = modp(W.lo[1] + y, nos) - nos / 2;
        int r = modp((-n / 2) * yv, nos);
        const int step = modp(yv, nos);
        T ar = T(0), ai = T(0);
        const C* c = Ci + (int64_t)x * n * n + kz;
#pragma unroll 4
        for (int ky = 0; ky < n; ky++) {
            cmac(c[(int64_t)ky * n], tw[r], 1, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        C o;
        o.x = ar;
        o.y = ai;
        E[idx] = o;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft3_i3(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const C* __restrict__ E = static_cast<const C*>(W.buf2);
    T* __restrict__ g = static_cast<T*>(W.grid);
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    const int n = W.n, nos = W.nos, By = W.B[1], Bz = W.B[2];
    const int64_t tot = (int64_t)W.B[0] * By * Bz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(idx % Bz);
        const int y = (int)((idx / Bz) % By);
        const int x = (int)(idx / ((int64_t)Bz * By));
        const int gz = modp(W.lo[2] + z, nos);
        const int zv = gz - nos / 2;
        int r = modp((-n / 2) * zv, nos);
        const int step = modp(zv, nos);
        const C* e = E + ((int64_t)x * By + y) * n;
        T ar = T(0);
#pragma unroll 4
        for (int kz = 0; kz < n; kz++) {
            const C v = e[kz];
            const C w = tw[r];
            // real part of v * conj(w)
            ar = fma(v.x, w.x, fma(v.y, w.y, ar));
            r += step;
            if (r >= nos) r -= nos;
        }
        g[((int64_t)modp(W.lo[0] + x, nos) * nos + modp(W.lo[1] + y, nos)) * nos + gz] = ar;
    }
}

// ---------------------------------------------------------------- slab form
// For boxes up to kSlab cells per axis: one CTA per x-slab runs F1 and F2 in
// shared memory (forward), one CTA per x-slab runs I2 and I3 (inverse); the
// middle pass is k_fft3_mid.  Three launches instead of five, and every line
// sum reads shared memory.
constexpr int kSlab = 64;
constexpr int kSlabThreads = 1024;

template <typename T, int NC = 0>
__global__ void __launch_bounds__(kSlabThreads) k_fft3_slab_fwd(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char slab_raw[];
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const int n = NC ? NC : W.n, nos = NC ? 2 * NC : W.nos, By = W.B[1], Bz = W.B[2];
    const int x = blockIdx.x;
    if (x >= W.B[0]) return;
    C* stw = reinterpret_cast<C*>(slab_raw);                  // nos twiddles
    T* P = reinterpret_cast<T*>(stw + nos);                   // By x Bz real plane
    C* Q = reinterpret_cast<C*>(P + ((By * Bz + 1) & ~1));    // By x n
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    for (int i = threadIdx.x; i < nos; i += blockDim.x) stw[i] = tw[i];
    const T* __restrict__ g = static_cast<const T*>(W.grid);
    const int gx = modp(W.lo[0] + x, nos);
    for (int i = threadIdx.x; i < By * Bz; i += blockDim.x) {
        const int y = i / Bz, z = i % Bz;
        P[i] = g[((int64_t)gx * nos + modp(W.lo[1] + y, nos)) * nos + modp(W.lo[2] + z, nos)];
    }
    __syncthreads();
    const int z0v = box_value0(W.lo[2], nos), y0v = box_value0(W.lo[1], nos);
    // this block's share of the kz columns (blockIdx.z of gridDim.z parts)
    const int ns = (n + gridDim.z - 1) / gridDim.z, kzb = blockIdx.z * ns, kze = min(n, kzb + ns);
    const int nc = kze - kzb;
    for (int i = threadIdx.x; i < By * nc; i += blockDim.x) {     // F1: z -> kz
        const int y = i / nc, kz = kzb + i % nc - n / 2;
        int r = modp(kz * z0v, nos);
        const int step = modp(kz, nos);
        T ar = T(0), ai = T(0);
        const T* prow = P + y * Bz;
#pragma unroll 4
        for (int z = 0; z < Bz; z++) {
            const C w = stw[r];
            ar = fma(prow[z], w.x, ar);
            ai = fma(prow[z], w.y, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        C o;
        o.x = ar;
        o.y = ai;
        Q[y * n + kz + n / 2] = o;
    }
    __syncthreads();
    C* __restrict__ Bo = static_cast<C*>(W.buf2);
    for (int i = threadIdx.x; i < n * nc; i += blockDim.x) {      // F2: y -> ky
        const int ky = i / nc - n / 2, kz = kzb + i % nc;
        int r = modp(ky * y0v, nos);
        const int step = modp(ky, nos);
        T ar = T(0), ai = T(0);
#pragma unroll 4
        for (int y = 0; y < By; y++) {
            cmac(Q[y * n + kz], stw[r], 0, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        C o;
        o.x = ar;
        o.y = ai;
        Bo[(int64_t)x * n * n + (ky + n / 2) * n + kz] = o;
    }
}

template <typename T, int NC = 0>
__global__ void __launch_bounds__(kSlabThreads) k_fft3_slab_inv(const Fft3Win* __restrict__ wins) {
    using C = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char slab_raw[];
    const Fft3Win W = wins[blockIdx.y];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const int n = NC ? NC : W.n, nos = NC ? 2 * NC : W.nos, By = W.B[1], Bz = W.B[2];
    const int x = blockIdx.x;
    if (x >= W.B[0]) return;
    C* stw = reinterpret_cast<C*>(slab_raw);       // nos twiddles
    C* Cs = stw + nos;                             // n x n
    C* E = Cs + n * n;                             // By x n
    const C* __restrict__ tw = static_cast<const C*>(W.tw);
    for (int i = threadIdx.x; i < nos; i += blockDim.x) stw[i] = tw[i];
    const C* __restrict__ Ci = static_cast<const C*>(W.buf1) + (int64_t)x * n * n;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Cs[i] = Ci[i];
    __syncthreads();
    // this block's share of the y rows (blockIdx.z of gridDim.z parts)
    const int ys = (By + gridDim.z - 1) / gridDim.z, yb = blockIdx.z * ys, ye = min(By, yb + ys);
    for (int i = threadIdx.x; i < (ye - yb) * n; i += blockDim.x) {   // I2: ky -> y
        const int y = yb + i / n, kz = i % n;
        const int yv = modp(W.lo[1] + y, nos) - nos / 2;
        int r = modp((-n / 2) * yv, nos);
        const int step = modp(yv, nos);
        T ar = T(0), ai = T(0);
#pragma unroll 4
        for (int ky = 0; ky < n; ky++) {
            cmac(Cs[ky * n + kz], stw[r], 1, ar, ai);
            r += step;
            if (r >= nos) r -= nos;
        }
        C o;
        o.x = ar;
        o.y = ai;
        E[y * n + kz] = o;
    }
    __syncthreads();
    T* __restrict__ g = static_cast<T*>(W.grid);
    const int gx = modp(W.lo[0] + x, nos);
    for (int i = threadIdx.x; i < (ye - yb) * Bz; i += blockDim.x) {  // I3: kz -> z, real part
        const int y = yb + i / Bz, z = i % Bz;
        const int gz = modp(W.lo[2] + z, nos);
        const int zv = gz - nos / 2;
        int r = modp((-n / 2) * zv, nos);
        const int step = modp(zv, nos);
        T ar = T(0);
        const C* e = E + y * n;
#pragma unroll 4
        for (int kz = 0; kz < n; kz++) {
            const C v = e[kz];
            const C w = stw[r];
            ar = fma(v.x, w.x, fma(v.y, w.y, ar));
            r += step;
            if (r >= nos) r -= nos;
        }
        g[((int64_t)gx * nos + modp(W.lo[1] + y, nos)) * nos + gz] = ar;
    }
}

template <typename T>
static size_t slab_fwd_bytes(int nos, int By, int Bz, int n) {
    using C = typename C2<T>::type;
    return nos * sizeof(C) + ((By * Bz + 1) & ~1) * sizeof(T) + (size_t)By * n * sizeof(C);
}
template <typename T>
static size_t slab_inv_bytes(int nos, int By, int n) {
    using C = typename C2<T>::type;
    return (nos + (size_t)n * n + (size_t)By * n) * sizeof(C);
}

bool fft3_box_supported(const WindowPlan& w) {
    return w.dA == 3 && w.n <= kMaxN3 && w.box_ext[0] <= kMaxBox3;
}

bool fft3_slab_supported(const WindowPlan& w) {
    return fft3_box_supported(w) && w.box_ext[1] <= kSlab && w.box_ext[2] <= kSlab && w.nos <= 4 * kSlab;
}

template <typename T>
static size_t mid_bytes() {
    using C = typename C2<T>::type;
    return ((size_t)(kMaxN3 + kMidStage) * kMidLanes + 4 * kMaxN3) * sizeof(C);
}

void Fft3Shape::add(const WindowPlan& w) {
    nw++;
    t1 = std::max<int64_t>(t1, (int64_t)w.box_ext[0] * w.box_ext[1] * w.n);
    t2 = std::max<int64_t>(t2, (int64_t)w.box_ext[0] * w.n * w.n);
    t3 = std::max<int64_t>(t3, (int64_t)w.box_ext[0] * w.box_ext[1] * w.box_ext[2]);
    nmax = std::max(nmax, w.n);
    nosmax = std::max(nosmax, w.nos);
    bx = std::max(bx, w.box_ext[0]);
    by = std::max(by, w.box_ext[1]);
    bz = std::max(bz, w.box_ext[2]);
    slab = slab && fft3_slab_supported(w);
    const int un = w.nos == 2 * w.n ? w.n : 0;
    uniform_n = (nw == 1) ? un : (uniform_n == un ? un : 0);
}

template <typename T, int NC>
static void launch_slab(const Fft3Win* wins, dim3 gs, dim3 gm, size_t shf, size_t shi, cudaStream_t st) {
    static bool attrs = [] {
        cudaFuncSetAttribute(k_fft3_slab_fwd<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_fft3_slab_inv<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_fft3_mid<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mid_bytes<T>());
        return true;
    }();
    (void)attrs;
    k_fft3_slab_fwd<T, NC><<<gs, kSlabThreads, shf, st>>>(wins);
    k_fft3_mid<T, NC><<<gm, kMidLanes * kMidWarps, mid_bytes<T>(), st>>>(wins);
    k_fft3_slab_inv<T, NC><<<gs, kSlabThreads, shi, st>>>(wins);
}

// every window of a descriptor array: one launch per pass for all of them
template <typename T>
anova_status fft3_box_run(const Fft3Win* wins, const Fft3Shape& sh, int sm_count, cudaStream_t st) {
    static bool mid_attr = [] {
        cudaFuncSetAttribute(k_fft3_mid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mid_bytes<T>());
        return true;
    }();
    (void)mid_attr;
    const int nw = sh.nw;
    if (nw == 0) return ANOVA_OK;
    const int cap = 4 * sm_count;
    const int nmax = sh.nmax;
    const dim3 g1(grid_for(sh.t1, kThreads, cap), nw), g2(grid_for(sh.t2, kThreads, cap), nw);
    const dim3 gm(nmax * ((nmax + kMidLanes - 1) / kMidLanes), nw), g3(grid_for(sh.t3, kThreads, cap), nw);
    if (sh.slab) {
        const size_t shf = slab_fwd_bytes<T>(sh.nosmax, sh.by, sh.bz, nmax);
        const size_t shi = slab_inv_bytes<T>(sh.nosmax, sh.by, nmax);
        const dim3 gs(sh.bx, nw, kSlabParts);
        switch (sh.uniform_n) {
            case 16: launch_slab<T, 16>(wins, gs, gm, shf, shi, st); break;
            case 32: launch_slab<T, 32>(wins, gs, gm, shf, shi, st); break;
            case 64: launch_slab<T, 64>(wins, gs, gm, shf, shi, st); break;
            default: launch_slab<T, 0>(wins, gs, gm, shf, shi, st); break;
        }
        ANOVA_CHECK_LAUNCH();
        return ANOVA_OK;
    }
    k_fft3_f1<T><<<g1, kThreads, 0, st>>>(wins);
    k_fft3_f2<T><<<g2, kThreads, 0, st>>>(wins);
    k_fft3_mid<T><<<gm, kMidLanes * kMidWarps, mid_bytes<T>(), st>>>(wins);
    k_fft3_i2<T><<<g1, kThreads, 0, st>>>(wins);
    k_fft3_i3<T><<<g3, kThreads, 0, st>>>(wins);
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template anova_status fft3_box_run<float>(const Fft3Win*, const Fft3Shape&, int, cudaStream_t);
template anova_status fft3_box_run<double>(const Fft3Win*, const Fft3Shape&, int, cudaStream_t);

// the plan's batched 3-D windows
template <typename T>
anova_status fft3_box_all(anova_plan* plan, cudaStream_t st) {
    const int nw = (int)plan->fft3_windows.size();
    if (nw == 0) return ANOVA_OK;
    Fft3Shape sh;
    for (int k = 0; k < nw; k++) sh.add(plan->win[plan->fft3_windows[k]]);
    sh.slab = plan->fft3_slab;
    return fft3_box_run<T>(plan->fft3_desc + (sizeof(T) == 8 ? 0 : nw), sh, plan->sm_count, st);
}

template anova_status fft3_box_all<float>(anova_plan*, cudaStream_t);
template anova_status fft3_box_all<double>(anova_plan*, cudaStream_t);

}  // namespace anova
