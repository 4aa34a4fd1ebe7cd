// dense3.cu -- spreading and gathering for 3-D windows as dense tensor-product
// sums over a bin's region (the window steps of the adjoint NFFT, Eq. adjnfft,
// and of the NFFT, Eq. nfft, in the fast summation of Sec. 4.2).
//
// Bins are Tb^3 grid cells (Tb = 2 or 4), so every node of a bin touches only the
// region of R = Tb + 2m <= 16 cells per axis starting at (bin * Tb - m).  Per node the window
// weights are zero-padded to that region:
//     wx[r] = psi(off_x + m + f_x - r),  r in [0, R)   (zero where |t| > m)
// so a node's contribution to the region is the outer product wx (x) wy (x) wz.
//
//   gather: one lane per node, the region of h staged in shared memory with a
//           row pitch of 16 along the last axis; every row is read with
//           broadcast 128-bit loads and contracted against the lane's own
//           weights:  s = sum_a wx[a] sum_b wy[b] sum_c wz[c] h[a][b][c].
//   spread: one thread per (a, pair of b, half of c) block of the region keeps
//           2 x 8 accumulators in registers and adds alpha_j wx wy wz for the
//           nodes of the sub-problem, whose weights are staged in shared
//           memory; the region is added to the global grid once at the end.
//
// Both loops are plain FP32 (or FP64) multiply-adds: no atomics per tap.
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"

namespace anova {

constexpr int kPitch = 16;        // shared row pitch along the last axis (elements)
constexpr int kGatherThreads = 256;
constexpr int kSpreadChunk = 64;  // nodes whose weights are staged at once

// Region cells bin*Tb - m + r lie in [-m, nos + Tb + m - 2], inside [-nos, 2 nos)
// because bin*Tb < nos, r < Tb + 2m and 2m + 2 <= nos, so one conditional add
// or subtract wraps them onto the torus.
__device__ __forceinline__ int wrap_idx(int u, int nos) {
    u += (u < 0) ? nos : 0;
    return u - ((u >= nos) ? nos : 0);
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    __device__ static __forceinline__ void load(const float* p, float* v) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};
template <>
struct Vec4<double> {
    __device__ static __forceinline__ void load(const double* p, double* v) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// ------------------------------------------------------------------ gather
template <typename T, int R>
__global__ void __launch_bounds__(kGatherThreads)
k_gather3_dense(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, DenseWin one, int m, T b,
                T norm, const float* __restrict__ poly) {
    static_assert(R <= kPitch, "region wider than the row pitch");
    constexpr bool kPoly = std::is_same<T, float>::value;
    __shared__ __align__(16) T reg[R * R * kPitch];
    __shared__ float sP[2 * 8 * kPsiStride];
    if (kPoly)
        for (int i = threadIdx.x; i < 2 * m * kPsiStride + 1; i += blockDim.x) sP[i] = poly[i];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs ? descs[sp.w] : one;
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const int32_t* __restrict__ perm = W.perm;
    const int32_t* __restrict__ cell = W.cell;
    const T* __restrict__ frac = static_cast<const T*>(W.frac);
    const T* __restrict__ h = static_cast<const T*>(W.grid);
    T* __restrict__ out = static_cast<T*>(W.out);
    const int64_t N = W.N;
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int ox = Tb * bx - m, oy = Tb * by - m, oz = Tb * bz - m;
    for (int i = threadIdx.x; i < R * R * kPitch; i += blockDim.x) {
        const int c = i % kPitch, ab = i / kPitch;
        const int bb = ab % R, a = ab / R;
        T v = T(0);
        if (c < R)
            v = h[((int64_t)wrap_idx(ox + a, nos) * nos + wrap_idx(oy + bb, nos)) * nos + wrap_idx(oz + c, nos)];
        reg[i] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const T mm = (T)m;
    for (int base = threadIdx.x - lane; base < sp.z; base += blockDim.x) {
        const int q = base + lane;
        const bool valid = q < sp.z;
        const int64_t pos = (int64_t)sp.y + (valid ? q : sp.z - 1);
        const T fx = frac[pos], fy = frac[N + pos], fz = frac[2 * N + pos];
        const int jx = cell[pos] - Tb * bx + m, jy = cell[N + pos] - Tb * by + m, jz = cell[2 * N + pos] - Tb * bz + m;
        const T tx = (T)jx + fx, ty = (T)jy + fy, tz = (T)jz + fz;
        // FP64 with the plan's tap table: the tap of region row r is k = r - (j - m), if in [0, 2m]
        const double* __restrict__ tp = (!kPoly && W.wtap) ? W.wtap + pos * 3 * (2 * m + 1) : nullptr;
        auto tap = [&](int t, int j, int r) -> T {
            const int k = r - j + m;
            return (k >= 0 && k <= 2 * m) ? (T)tp[t * (2 * m + 1) + k] : T(0);
        };
        T wy[R], wz[kPitch];
#pragma unroll
        for (int r = 0; r < R; r++)
            wy[r] = kPoly ? (T)psi_poly_eval(sP, jy - r, (float)fy, m)
                          : (tp ? tap(1, jy, r) : kb_psi<T>(ty - (T)r, mm, b, norm));
#pragma unroll
        for (int r = 0; r < kPitch; r++)
            wz[r] = (r < R) ? (kPoly ? (T)psi_poly_eval(sP, jz - r, (float)fz, m)
                                     : (tp ? tap(2, jz, r) : kb_psi<T>(tz - (T)r, mm, b, norm)))
                            : T(0);
        T acc = T(0);
#pragma unroll 1
        for (int a = 0; a < R; a++) {
            const T wa = kPoly ? (T)psi_poly_eval(sP, jx - a, (float)fx, m)
                               : (tp ? tap(0, jx, a) : kb_psi<T>(tx - (T)a, mm, b, norm));
            const T* rows = reg + a * R * kPitch;
            T sa = T(0);
#pragma unroll
            for (int bb = 0; bb < R; bb++) {
                const T* row = rows + bb * kPitch;
                T s = T(0);
#pragma unroll
                for (int c4 = 0; c4 < (R + 3) / 4; c4++) {
                    T v[4];
                    Vec4<T>::load(row + 4 * c4, v);
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (4 * c4 + k < R) s = fma(wz[4 * c4 + k], v[k], s);
                }
                sa = fma(wy[bb], s, sa);
            }
            acc = fma(wa, sa, acc);
        }
        if (valid) out[perm[pos]] = acc;
    }
}

// ------------------------------------------------------------------ spread
template <typename T, int R>
__global__ void __launch_bounds__(R * (R / 2 + R % 2) * 2)
k_spread3_dense(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, DenseWin one,
                const void* __restrict__ alpha, int alpha_double, int m, T b, T norm,
                const float* __restrict__ poly) {
    constexpr bool kPoly = std::is_same<T, float>::value;
    __shared__ float sP[2 * 8 * kPsiStride];
    static_assert(R <= kPitch, "region wider than the row pitch");
    constexpr int BP = R / 2 + R % 2;          // pairs of b rows
    constexpr int NT = R * BP * 2;             // threads: a x b-pair x c-half
    __shared__ __align__(16) T wxs[kSpreadChunk][R];
    __shared__ __align__(16) T wys[kSpreadChunk][kPitch];
    __shared__ __align__(16) T wzs[kSpreadChunk][kPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs ? descs[sp.w] : one;
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const int32_t* __restrict__ perm = W.perm;
    const int32_t* __restrict__ cell = W.cell;
    const T* __restrict__ frac = static_cast<const T*>(W.frac);
    T* __restrict__ grid = static_cast<T*>(W.grid);
    const int64_t N = W.N;
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int tid = threadIdx.x;
    const int ch = tid & 1, bp = (tid >> 1) % BP, a = (tid >> 1) / BP;
    const int b0 = 2 * bp, c0 = 8 * ch;
    const T mm = (T)m;
    T acc[2][8];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 8; k++) acc[i][k] = T(0);

    if (kPoly)
        for (int i = tid; i < 2 * m * kPsiStride + 1; i += NT) sP[i] = poly[i];
    for (int first = 0; first < sp.z; first += kSpreadChunk) {
        const int cnt = min(kSpreadChunk, sp.z - first);
        __syncthreads();
        // stage the weights of `cnt` nodes: 3 axes x kPitch entries each
        for (int i = tid; i < cnt * 3 * kPitch; i += NT) {
            const int r = i % kPitch, ax = (i / kPitch) % 3, p = i / (3 * kPitch);
            const int64_t pos = (int64_t)sp.y + first + p;
            const int bcoord = (ax == 0) ? bx : (ax == 1) ? by : bz;
            const int j = cell[ax * N + pos] - Tb * bcoord + m - r;
            T w = T(0);
            if (r < R) {
                if (!kPoly && W.wtap) {
                    // FP64 with the plan's tap table: j = m - k for tap k
                    const int k = m - j;
                    w = (k >= 0 && k <= 2 * m) ? (T)W.wtap[(pos * 3 + ax) * (2 * m + 1) + k] : T(0);
                } else {
                    const T f = frac[ax * N + pos];
                    w = kPoly ? (T)psi_poly_eval(sP, j, (float)f, m) : kb_psi<T>((T)j + f, mm, b, norm);
                }
            }
            if (ax == 0) {
                if (r < R) {
                    const int32_t src = perm[pos];
                    const T al = alpha_double ? (T)(static_cast<const double*>(alpha)[src])
                                              : (T)(static_cast<const float*>(alpha)[src]);
                    wxs[p][r] = al * w;
                }
            } else if (ax == 1) {
                wys[p][r] = w;
            } else {
                wzs[p][r] = w;
            }
        }
        __syncthreads();
        if (a < R) {
            for (int p = 0; p < cnt; p++) {
                const T wa = wxs[p][a];
                const T w0 = wa * wys[p][b0];
                const T w1 = wa * wys[p][b0 + 1];
                T z[8];
                Vec4<T>::load(&wzs[p][c0], z);
                Vec4<T>::load(&wzs[p][c0 + 4], z + 4);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    acc[0][k] = fma(w0, z[k], acc[0][k]);
                    acc[1][k] = fma(w1, z[k], acc[1][k]);
                }
            }
        }
    }
    if (a < R) {
        const int ga = wrap_idx(Tb * bx - m + a, nos);
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int bb = b0 + i;
            if (bb >= R) continue;
            const int64_t rowbase = ((int64_t)ga * nos + wrap_idx(Tb * by - m + bb, nos)) * nos;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int c = c0 + k;
                if (c < R) atomicAdd(&grid[rowbase + wrap_idx(Tb * bz - m + c, nos)], acc[i][k]);
            }
        }
    }
}

// --------------------------------------------------- FP32 with weight table
// Packed FP32 multiply-add / multiply on (x, y) pairs (Blackwell f32x2 instructions).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Gather, FP32, weights read from the plan's table.  Every lane handles two
// nodes of the bin; each row h[a][b][:] is read once (broadcast) and
// contracted against both nodes' z weights (packed FMA), then
// s += wx[a] wy[b] (row . wz) per node.
constexpr int kGather2Threads = 128;
template <int R>
__global__ void __launch_bounds__(kGather2Threads, 3)
k_gather3_f32(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m) {
    static_assert(R <= kPitch && R % 2 == 0, "even region up to the row pitch");
    constexpr int RP = R / 2;                      // c-pairs per row
    constexpr int NV = (R + 3) / 4;                // float4 per row
    __shared__ __align__(16) float reg[R * R * kPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const float* __restrict__ h = static_cast<const float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int ox = Tb * bx - m, oy = Tb * by - m, oz = Tb * bz - m;
    {
        // thread -> (row, c) with c fastest: one wrapped row base per row
        const int c = threadIdx.x % kPitch;
        const int gz = wrap_idx(oz + c, nos);
        for (int ab = threadIdx.x / kPitch; ab < R * R; ab += blockDim.x / kPitch) {
            const int a = ab / R, bb = ab - a * R;
            float v = 0.f;
            if (c < R) v = h[(wrap_idx(ox + a, nos) * nos + wrap_idx(oy + bb, nos)) * nos + gz];
            reg[ab * kPitch + c] = v;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* __restrict__ out = static_cast<float*>(W.out);
    for (int base = warp * 64; base < sp.z; base += (kGather2Threads / 32) * 64) {
        const int q0 = base + lane, q1 = base + 32 + lane;
        const bool v0 = q0 < sp.z, v1 = q1 < sp.z;
        const int64_t p0 = (int64_t)sp.y + (v0 ? q0 : sp.z - 1);
        const int64_t p1 = (int64_t)sp.y + (v1 ? q1 : sp.z - 1);
        float wy0[R], wy1[R];
        float2 wz0[RP], wz1[RP];
        {
            const float* a0 = W.wtab + p0 * 48;
            const float* a1 = W.wtab + p1 * 48;
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const float4 y0 = reinterpret_cast<const float4*>(a0 + 16)[k];
                const float4 y1 = reinterpret_cast<const float4*>(a1 + 16)[k];
                const float4 z0 = reinterpret_cast<const float4*>(a0 + 32)[k];
                const float4 z1 = reinterpret_cast<const float4*>(a1 + 32)[k];
                const float ya[4] = {y0.x, y0.y, y0.z, y0.w}, yb[4] = {y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (4 * k + e < R) { wy0[4 * k + e] = ya[e]; wy1[4 * k + e] = yb[e]; }
                if (2 * k < RP) { wz0[2 * k] = make_float2(z0.x, z0.y); wz1[2 * k] = make_float2(z1.x, z1.y); }
                if (2 * k + 1 < RP) { wz0[2 * k + 1] = make_float2(z0.z, z0.w); wz1[2 * k + 1] = make_float2(z1.z, z1.w); }
            }
        }
        const float* __restrict__ wx0 = W.wtab + p0 * 48;
        const float* __restrict__ wx1 = W.wtab + p1 * 48;
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 1
        for (int a = 0; a < R; a++) {
            const float4* rows = reinterpret_cast<const float4*>(reg + a * R * kPitch);
            float sa0 = 0.f, sa1 = 0.f;
#pragma unroll
            for (int bb = 0; bb < R; bb++) {
                float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int c4 = 0; c4 < NV; c4++) {
                    const float4 v = rows[bb * (kPitch / 4) + c4];
                    if (2 * c4 < RP) {
                        const float2 hv = make_float2(v.x, v.y);
                        s0 = ffma2(wz0[2 * c4], hv, s0);
                        s1 = ffma2(wz1[2 * c4], hv, s1);
                    }
                    if (2 * c4 + 1 < RP) {
                        const float2 hv = make_float2(v.z, v.w);
                        s0 = ffma2(wz0[2 * c4 + 1], hv, s0);
                        s1 = ffma2(wz1[2 * c4 + 1], hv, s1);
                    }
                }
                sa0 = fmaf(wy0[bb], s0.x + s0.y, sa0);
                sa1 = fmaf(wy1[bb], s1.x + s1.y, sa1);
            }
            acc0 = fmaf(__ldg(wx0 + a), sa0, acc0);
            acc1 = fmaf(__ldg(wx1 + a), sa1, acc1);
        }
        if (v0) out[W.perm[p0]] = acc0;
        if (v1) out[W.perm[p1]] = acc1;
    }
}

// asort_w[pos] = alpha[perm_w[pos]] for every dense window (one launch), so
// that the spread reads its coefficients contiguously with the weight rows.
__global__ void k_sort_alpha(const DenseWin* __restrict__ descs, int nd, int64_t N, const void* __restrict__ alpha,
                             int alpha_double) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N * nd;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx / N);
        const int64_t pos = idx - (int64_t)w * N;
        const DenseWin& W = descs[w];
        const int32_t src = W.perm[pos];
        W.asort[pos] = alpha_double ? (float)(static_cast<const double*>(alpha)[src])
                                    : static_cast<const float*>(alpha)[src];
    }
}

// Spread, FP32, weights read from the plan's table.  Thread (a, b-pair,
// c-half) keeps its 2 x 8 region cells as packed pairs.  x and y weights are
// staged as duplicated pairs so that the per-node products are packed
// multiplies; the next chunk's table rows are fetched into registers while
// the current chunk is accumulated.
template <int R>
__global__ void __launch_bounds__(R * (R / 2) * 2)
k_spread3_f32(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, const void* __restrict__ alpha,
              int alpha_double, int m) {
    static_assert(R <= kPitch && R % 2 == 0, "even region up to the row pitch");
    constexpr int BP = R / 2;
    constexpr int NT = R * BP * 2;
    constexpr int PER = (kSpreadChunk * 12 + NT - 1) / NT;   // float4 table entries per thread per chunk
    __shared__ __align__(16) float2 wxs[kSpreadChunk][kPitch];   // (alpha wx, alpha wx)
    __shared__ __align__(16) float2 wys[kSpreadChunk][kPitch];   // (wy, wy)
    __shared__ __align__(16) float wzs[kSpreadChunk][kPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    float* __restrict__ grid = static_cast<float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int tid = threadIdx.x;
    const int ch = tid & 1, bp = (tid >> 1) % BP, a = (tid >> 1) / BP;
    const int b0 = 2 * bp, c0 = 8 * ch;
    float2 acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int k = 0; k < 4; k++) acc[i][k] = make_float2(0.f, 0.f);

    float4 pre[PER];
    float pal[PER];
    auto fetch = [&](int first) {
        const int cnt = min(kSpreadChunk, sp.z - first);
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int i = tid + u * NT;
            pre[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            pal[u] = 0.f;
            if (i < cnt * 12) {
                const int p = i / 12, k = i % 12;
                const int64_t pos = (int64_t)sp.y + first + p;
                pre[u] = reinterpret_cast<const float4*>(W.wtab + pos * 48)[k];
                if (k < 4) pal[u] = W.asort[pos];
            }
        }
    };
    auto stage = [&](int first) {
        const int cnt = min(kSpreadChunk, sp.z - first);
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int i = tid + u * NT;
            if (i < cnt * 12) {
                const int p = i / 12, k = i % 12;
                float4 v = pre[u];
                if (k < 4) {
                    const float al = pal[u];
                    float4* d = reinterpret_cast<float4*>(&wxs[p][4 * k]);
                    d[0] = make_float4(al * v.x, al * v.x, al * v.y, al * v.y);
                    d[1] = make_float4(al * v.z, al * v.z, al * v.w, al * v.w);
                } else if (k < 8) {
                    float4* d = reinterpret_cast<float4*>(&wys[p][4 * (k - 4)]);
                    d[0] = make_float4(v.x, v.x, v.y, v.y);
                    d[1] = make_float4(v.z, v.z, v.w, v.w);
                } else {
                    reinterpret_cast<float4*>(wzs[p])[k - 8] = v;
                }
            }
        }
    };
    fetch(0);
    for (int first = 0; first < sp.z; first += kSpreadChunk) {
        const int cnt = min(kSpreadChunk, sp.z - first);
        __syncthreads();
        stage(first);
        __syncthreads();
        if (first + kSpreadChunk < sp.z) fetch(first + kSpreadChunk);
#pragma unroll 2
        for (int p = 0; p < cnt; p++) {
            const float2 wa = wxs[p][a];
            const float4 wy = *reinterpret_cast<const float4*>(&wys[p][b0]);
            const float4 z0 = *reinterpret_cast<const float4*>(&wzs[p][c0]);
            const float4 z1 = *reinterpret_cast<const float4*>(&wzs[p][c0 + 4]);
            const float2 W0 = fmul2(wa, make_float2(wy.x, wy.y));
            const float2 W1 = fmul2(wa, make_float2(wy.z, wy.w));
            const float2 z[4] = {make_float2(z0.x, z0.y), make_float2(z0.z, z0.w), make_float2(z1.x, z1.y),
                                 make_float2(z1.z, z1.w)};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                acc[0][k] = ffma2(W0, z[k], acc[0][k]);
                acc[1][k] = ffma2(W1, z[k], acc[1][k]);
            }
        }
    }
    const int ga = wrap_idx(Tb * bx - m + a, nos);
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int64_t rowbase = ((int64_t)ga * nos + wrap_idx(Tb * by - m + b0 + i, nos)) * nos;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int c = c0 + 2 * k;
            if (c < R) atomicAdd(&grid[rowbase + wrap_idx(Tb * bz - m + c, nos)], acc[i][k].x);
            if (c + 1 < R) atomicAdd(&grid[rowbase + wrap_idx(Tb * bz - m + c + 1, nos)], acc[i][k].y);
        }
    }
}

// ------------------------------------------------- tensor-core spread (TF32)
// The spread of one sub-problem is the product C[(a,b), c] = sum_p A[(a,b), p]
// B[p, c] with A = wx (x) wy and B = alpha wz: a dense contraction over the
// nodes of the bin, run on mma.sync m16n8k8 TF32.  FP32 accuracy comes from
// splitting every operand into a TF32 head and a tail and accumulating
// head*head + head*tail + tail*head in FP32 (the dropped tail*tail term is
// 2^-22 relative).  The tail is passed as the FP32 residual x - head: the
// tensor core reads only its TF32 bits (rounding toward zero, 2^-21 relative
// to x).  Warp w owns the M-tiles a = 2w, 2w+1 (16 b-rows each) and both
// N-tiles (c = 0..7, 8..15), so every accumulator pair of a thread is two
// neighbouring cells along the grid's last axis: one 8-byte atomic each.
__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_of(x);
    lo = tf32_of(x - __uint_as_float(hi));
}
__device__ __forceinline__ void tf32_split_fast(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_of(x);
    lo = __float_as_uint(x - __uint_as_float(hi));
}
// head by truncation to TF32's 10 mantissa bits (one logic operation), tail
// the exact FP32 residual x - head (at most 2^-10 |x|; the tensor core reads
// its TF32 bits, so the pair keeps x to 2^-20 relative)
__device__ __forceinline__ void tf32_split_trunc(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kTcPitch = 24;   // shared row pitch: rows p and p+1..3 land in distinct bank groups
template <int R>
__global__ void __launch_bounds__(32 * ((R + 1) / 2))
k_spread3_tc(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m,
             const void* __restrict__ alpha = nullptr, int alpha_double = 0) {
    static_assert(R <= kPitch && R % 2 == 0, "even region up to 16");
    constexpr int NW = R / 2;                  // warps, two a-tiles each
    constexpr int NT = 32 * NW;
    __shared__ __align__(16) uint32_t szh[kSpreadChunk][kTcPitch];   // alpha wz, TF32 head
    __shared__ __align__(16) uint32_t szl[kSpreadChunk][kTcPitch];   // and tail
    __shared__ __align__(16) float sx[kSpreadChunk][kTcPitch];
    __shared__ __align__(16) float sy[kSpreadChunk][kTcPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    float* __restrict__ grid = static_cast<float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.f;
    for (int first = 0; first < sp.z; first += kSpreadChunk) {
        const int cnt = min(kSpreadChunk, sp.z - first);
        const int cnt8 = (cnt + 7) & ~7;
        __syncthreads();
        for (int i = tid; i < cnt8 * 12; i += NT) {
            const int p = i / 12, k = i % 12;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            float al = 0.f;
            if (p < cnt) {
                const int64_t pos = (int64_t)sp.y + first + p;
                v = reinterpret_cast<const float4*>(W.wtab + pos * 48)[k];
                // the coefficient of the node: gathered through the permutation from the
                // caller's vector (L2-resident), or the sorted copy of a batch instance
                if (k >= 8)
                    al = !alpha ? W.asort[pos]
                                : alpha_double ? (float)static_cast<const double*>(alpha)[W.perm[pos]]
                                               : static_cast<const float*>(alpha)[W.perm[pos]];
            }
            if (k < 4) {
                *reinterpret_cast<float4*>(&sx[p][4 * k]) = v;
            } else if (k < 8) {
                *reinterpret_cast<float4*>(&sy[p][4 * (k - 4)]) = v;
            } else {
                const float zs[4] = {al * v.x, al * v.y, al * v.z, al * v.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    uint32_t hi, lo;
                    tf32_split_fast(zs[e], hi, lo);
                    szh[p][4 * (k - 8) + e] = hi;
                    szl[p][4 * (k - 8) + e] = lo;
                }
            }
        }
        __syncthreads();
        for (int p0 = 0; p0 < cnt8; p0 += 8) {
            const int pa = p0 + t, pb = p0 + t + 4;
            const float y0 = sy[pa][g], y1 = sy[pa][g + 8], y2 = sy[pb][g], y3 = sy[pb][g + 8];
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                bh[nt][0] = szh[pa][8 * nt + g];
                bl[nt][0] = szl[pa][8 * nt + g];
                bh[nt][1] = szh[pb][8 * nt + g];
                bl[nt][1] = szl[pb][8 * nt + g];
            }
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int a = 2 * warp + i;
                const float x0 = sx[pa][a], x1 = sx[pb][a];
                uint32_t ah[4], alo[4];
                tf32_split_fast(x0 * y0, ah[0], alo[0]);
                tf32_split_fast(x0 * y1, ah[1], alo[1]);
                tf32_split_fast(x1 * y2, ah[2], alo[2]);
                tf32_split_fast(x1 * y3, ah[3], alo[3]);
#pragma unroll
                for (int nt = 0; nt < 2; nt++) {
                    mma_tf32(acc[i][nt], ah, bh[nt][0], bh[nt][1]);
                    mma_tf32(acc[i][nt], ah, bl[nt][0], bl[nt][1]);
                    mma_tf32(acc[i][nt], alo, bh[nt][0], bh[nt][1]);
                }
            }
        }
    }
    // acc[i][nt] holds C rows b = g (e = 0, 1) and b = g + 8 (e = 2, 3), columns
    // c = 8 nt + 2t (e even) and c + 1 (e odd) of the M-tile a = 2 warp + i.
    // A pair goes out as one float2 atomic when its first cell is 8-byte aligned
    // (an aligned grid and an even index; nos is even, so c + 1 does not wrap).
    const bool vec_ok = (reinterpret_cast<uintptr_t>(grid) & 7) == 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int a = 2 * warp + i;
        const int ga = wrap_idx(Tb * bx - m + a, nos);
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int b = g + 8 * h;
                const int c = 8 * nt + 2 * t;
                if (b < R && c < R) {
                    const int row = (ga * nos + wrap_idx(Tb * by - m + b, nos)) * nos;
                    const int gc = wrap_idx(Tb * bz - m + c, nos);
                    const float v0 = acc[i][nt][2 * h], v1 = acc[i][nt][2 * h + 1];
                    if (vec_ok && (gc & 1) == 0 && gc + 1 < nos) {
                        atomicAdd(reinterpret_cast<float2*>(&grid[row + gc]), make_float2(v0, v1));
                    } else {
                        atomicAdd(&grid[row + gc], v0);
                        atomicAdd(&grid[row + wrap_idx(Tb * bz - m + c + 1, nos)], v1);
                    }
                }
            }
    }
}

// The same spread with the staging pipelined: while the MMAs of chunk k run,
// cp.async copies chunk k + 1's weight-table rows and coefficients into the
// other of two shared buffers (raw rows: x weights 0..15, y 16..31, z 32..47).
// Per chunk: wait for its copies, one barrier, start the next chunk's copies,
// form (alpha wz) as TF32 head and tail, a second barrier, the MMAs.  The
// node permutation is read one chunk ahead into a register, so the coefficient
// copy (through the permutation) does not wait for it.
constexpr int kTpPitch = 56;   // floats per staged row: 224 bytes, conflict-free fragment reads

__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

template <int R>
__global__ void __launch_bounds__(32 * (R / 2), (R <= 14 ? 5 : 4))
k_spread3_tcp(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m,
              const void* __restrict__ alpha = nullptr, int alpha_double = 0) {
    static_assert(R <= kPitch && R % 2 == 0, "even region up to 16");
    constexpr int NW = R / 2;
    constexpr int NT = 32 * NW;
    __shared__ __align__(16) float raw[2][kSpreadChunk][kTpPitch];
    __shared__ __align__(16) double sal[2][kSpreadChunk];             // coefficients as copied (FP32 or FP64)
    __shared__ __align__(16) uint32_t szh[kSpreadChunk][kTcPitch];   // alpha wz, TF32 head
    __shared__ __align__(16) uint32_t szl[kSpreadChunk][kTcPitch];   // and tail
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    float* __restrict__ grid = static_cast<float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const bool dbl = alpha && alpha_double;
    // copies of chunk [first, first + cnt) into buffer b; `pm` is the permutation entry of node
    // first + tid (tid < cnt) when the coefficients come through the permutation
    auto stage = [&](int b, int first, int32_t pm) {
        const int cnt = min(kSpreadChunk, sp.z - first);
        for (int i = tid; i < cnt * 12; i += NT) {
            const int p = i / 12, k = i % 12;
            cp_async_16(&raw[b][p][4 * k], W.wtab + ((int64_t)sp.y + first + p) * 48 + 4 * k);
        }
        if (tid < cnt) {
            const int64_t pos = (int64_t)sp.y + first + tid;
            if (!alpha) cp_async_4(&sal[b][tid], W.asort + pos);
            else if (dbl) cp_async_8(&sal[b][tid], static_cast<const double*>(alpha) + pm);
            else cp_async_4(&sal[b][tid], static_cast<const float*>(alpha) + pm);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto perm_of = [&](int first) -> int32_t {
        return (alpha && first + tid < sp.z && tid < kSpreadChunk) ? W.perm[(int64_t)sp.y + first + tid] : 0;
    };
    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.f;
    stage(0, 0, perm_of(0));
    int32_t pnext = perm_of(kSpreadChunk);
    int b = 0;
    for (int first = 0; first < sp.z; first += kSpreadChunk, b ^= 1) {
        const int cnt = min(kSpreadChunk, sp.z - first);
        const int cnt8 = (cnt + 7) & ~7;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();          // chunk `first` is in buffer b; the MMAs of the previous chunk are done
        if (first + kSpreadChunk < sp.z) {
            stage(b ^ 1, first + kSpreadChunk, pnext);
            pnext = perm_of(first + 2 * kSpreadChunk);
        }
        for (int i = tid; i < cnt8 * 16; i += NT) {
            const int p = i >> 4, e = i & 15;
            uint32_t hi = 0u, lo = 0u;
            if (p < cnt) {
                const float al = dbl ? (float)sal[b][p] : reinterpret_cast<const float*>(&sal[b][p])[0];
                tf32_split_trunc(al * raw[b][p][32 + e], hi, lo);
            } else {
                raw[b][p][e] = 0.f;
                raw[b][p][16 + e] = 0.f;
            }
            szh[p][e] = hi;
            szl[p][e] = lo;
        }
        __syncthreads();
        for (int p0 = 0; p0 < cnt8; p0 += 8) {
            const int pa = p0 + t, pb = p0 + t + 4;
            const float y0 = raw[b][pa][16 + g], y1 = raw[b][pa][24 + g], y2 = raw[b][pb][16 + g],
                        y3 = raw[b][pb][24 + g];
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                bh[nt][0] = szh[pa][8 * nt + g];
                bl[nt][0] = szl[pa][8 * nt + g];
                bh[nt][1] = szh[pb][8 * nt + g];
                bl[nt][1] = szl[pb][8 * nt + g];
            }
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int a = 2 * warp + i;
                const float x0 = raw[b][pa][a], x1 = raw[b][pb][a];
                uint32_t ah[4], alo[4];
                tf32_split_trunc(x0 * y0, ah[0], alo[0]);
                tf32_split_trunc(x0 * y1, ah[1], alo[1]);
                tf32_split_trunc(x1 * y2, ah[2], alo[2]);
                tf32_split_trunc(x1 * y3, ah[3], alo[3]);
#pragma unroll
                for (int nt = 0; nt < 2; nt++) {
                    mma_tf32(acc[i][nt], ah, bh[nt][0], bh[nt][1]);
                    mma_tf32(acc[i][nt], ah, bl[nt][0], bl[nt][1]);
                    mma_tf32(acc[i][nt], alo, bh[nt][0], bh[nt][1]);
                }
            }
        }
    }
    // flush as in k_spread3_tc
    const bool vec_ok = (reinterpret_cast<uintptr_t>(grid) & 7) == 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int a = 2 * warp + i;
        const int ga = wrap_idx(Tb * bx - m + a, nos);
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int bb = g + 8 * h;
                const int c = 8 * nt + 2 * t;
                if (bb < R && c < R) {
                    const int row = (ga * nos + wrap_idx(Tb * by - m + bb, nos)) * nos;
                    const int gc = wrap_idx(Tb * bz - m + c, nos);
                    const float v0 = acc[i][nt][2 * h], v1 = acc[i][nt][2 * h + 1];
                    if (vec_ok && (gc & 1) == 0 && gc + 1 < nos) {
                        atomicAdd(reinterpret_cast<float2*>(&grid[row + gc]), make_float2(v0, v1));
                    } else {
                        atomicAdd(&grid[row + gc], v0);
                        atomicAdd(&grid[row + wrap_idx(Tb * bz - m + c + 1, nos)], v1);
                    }
                }
            }
    }
}

// ------------------------------------------------- tensor-core gather (TF32)
// Per warp, 16 nodes j of the bin: U[j][(a,b)] = sum_c wz_j[c] h[a][b][c] on
// mma.sync m16n8k8 TF32 (A = the nodes' z weights, B = rows of the staged
// region, 3xTF32 for FP32 accuracy), then s_j = sum_a wx_j[a] sum_b wy_j[b]
// U[j][(a,b)] on the accumulator fragments and a reduction over the 4 lanes
// that share a node.  The region is staged once per CTA as TF32 heads and
// tails with a 20-float row pitch (conflict-free fragment loads).
constexpr int kTcRowPitch = 20;
constexpr int kGatherTcThreads = 128;
template <int R>
__global__ void __launch_bounds__(kGatherTcThreads)
k_gather3_tc(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m) {
    static_assert(R <= kPitch && R % 2 == 0, "even region up to 16");
    __shared__ __align__(16) uint32_t rh[R * R * kTcRowPitch];
    __shared__ __align__(16) uint32_t rl[R * R * kTcRowPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const float* __restrict__ h = static_cast<const float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int ox = Tb * bx - m, oy = Tb * by - m, oz = Tb * bz - m;
    {
        const int c = threadIdx.x % kPitch;
        const int gz = wrap_idx(oz + c, nos);
        for (int ab = threadIdx.x / kPitch; ab < R * R; ab += blockDim.x / kPitch) {
            const int a = ab / R, bb = ab - a * R;
            float v = 0.f;
            if (c < R) v = h[(wrap_idx(ox + a, nos) * nos + wrap_idx(oy + bb, nos)) * nos + gz];
            uint32_t hi, lo;
            tf32_split(v, hi, lo);
            rh[ab * kTcRowPitch + c] = hi;
            rl[ab * kTcRowPitch + c] = lo;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    float* __restrict__ out = static_cast<float*>(W.out);
    for (int base = warp * 16; base < sp.z; base += (kGatherTcThreads / 32) * 16) {
        const int j0 = base + g, j1 = base + g + 8;
        const bool v0 = j0 < sp.z, v1 = j1 < sp.z;
        const int64_t p0 = (int64_t)sp.y + (v0 ? j0 : sp.z - 1);
        const int64_t p1 = (int64_t)sp.y + (v1 ? j1 : sp.z - 1);
        const float* w0 = W.wtab + p0 * 48;
        const float* w1 = W.wtab + p1 * 48;
        // A fragments for the two k-steps (c = 0..7, 8..15): a0 (j0, t), a1 (j1, t), a2 (j0, t+4), a3 (j1, t+4)
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            tf32_split(v0 ? __ldg(w0 + 32 + 8 * ks + t) : 0.f, ah[ks][0], al[ks][0]);
            tf32_split(v1 ? __ldg(w1 + 32 + 8 * ks + t) : 0.f, ah[ks][1], al[ks][1]);
            tf32_split(v0 ? __ldg(w0 + 32 + 8 * ks + t + 4) : 0.f, ah[ks][2], al[ks][2]);
            tf32_split(v1 ? __ldg(w1 + 32 + 8 * ks + t + 4) : 0.f, ah[ks][3], al[ks][3]);
        }
        // y weights at the fragment columns b = 8 nt + 2t, 8 nt + 2t + 1; x weights of both nodes
        float y0[2][2], y1[2][2], x0[R], x1[R];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int b = 8 * nt + 2 * t + e;
                y0[nt][e] = (b < R) ? __ldg(w0 + 16 + b) : 0.f;
                y1[nt][e] = (b < R) ? __ldg(w1 + 16 + b) : 0.f;
            }
#pragma unroll
        for (int a = 0; a < R; a++) {
            x0[a] = __ldg(w0 + a);
            x1[a] = __ldg(w1 + a);
        }
        float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
        for (int a = 0; a < R; a++) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                if (8 * nt >= R) continue;
                // head*head and the two correction products accumulate separately
                float ch[4] = {0.f, 0.f, 0.f, 0.f}, cx[4] = {0.f, 0.f, 0.f, 0.f};
                const int brow = a * R + 8 * nt + g;          // B column n = b = 8 nt + g
                const bool brow_ok = 8 * nt + g < R;
#pragma unroll
                for (int ks = 0; ks < 2; ks++) {
                    uint32_t bh0 = 0, bh1 = 0, bl0 = 0, bl1 = 0;
                    if (brow_ok) {
                        const int o = brow * kTcRowPitch + 8 * ks + t;
                        bh0 = rh[o];
                        bh1 = rh[o + 4];
                        bl0 = rl[o];
                        bl1 = rl[o + 4];
                    }
                    mma_tf32(ch, ah[ks], bh0, bh1);
                    mma_tf32(cx, ah[ks], bl0, bl1);
                    mma_tf32(cx, al[ks], bh0, bh1);
                }
                s0 = fmaf(y0[nt][0], ch[0] + cx[0], fmaf(y0[nt][1], ch[1] + cx[1], s0));
                s1 = fmaf(y1[nt][0], ch[2] + cx[2], fmaf(y1[nt][1], ch[3] + cx[3], s1));
            }
            acc0 = fmaf(x0[a], s0, acc0);
            acc1 = fmaf(x1[a], s1, acc1);
        }
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, 1);
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, 2);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, 1);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, 2);
        if (t == 0) {
            if (v0) out[W.perm[p0]] = acc0;
            if (v1) out[W.perm[p1]] = acc1;
        }
    }
}

// ------------------------------------------------ 2-D and 1-D windows, FP32
// Same binning and weight table as the 3-D kernels (rows of 16 floats per axis),
// regions R x R (2-D, bins of 2x2 cells) and R (1-D).  The work per node is small
// (R^2 or R multiply-adds), so one warp accumulates a sub-problem's region in
// registers and adds it to the grid once, and the gather is one thread per node.

// 2-D spread: a block of kGroupWarps warps takes as many consecutive
// sub-problems, one per warp; lane (a = lane/2, half h) keeps cells
// (a, 8h .. 8h+7) of its warp's region.  Warps whose sub-problems share a bin
// (consecutive in the list) add their regions in shared memory and the first
// of them adds the sum to the grid: with many nodes per cell the grid atomics,
// contended by every sub-problem of the neighbouring bins, are the cost.
constexpr int kGroupWarps = 8;
constexpr int kGroupChunk = 32;            // nodes staged per warp at a time

template <int R>
__global__ void __launch_bounds__(32 * kGroupWarps) k_spread2_f32(const int4* __restrict__ sub,
                                                                  const DenseWin* __restrict__ descs, int m,
                                                                  int nsub) {
    static_assert(R <= kPitch, "region up to 16");
    __shared__ __align__(16) float sx[kGroupWarps][kGroupChunk][kPitch];
    __shared__ __align__(16) float sy[kGroupWarps][kGroupChunk][kPitch];
    __shared__ __align__(16) float red[kGroupWarps][16][16];
    __shared__ int key[kGroupWarps][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = lane >> 1, h = lane & 1;
    const int si = blockIdx.x * kGroupWarps + warp;
    int4 sp = make_int4(0, 0, 0, 0);
    bool active = si < nsub;
    if (active) sp = sub[si];
    const DenseWin W = descs[active ? sp.w : sub[blockIdx.x * kGroupWarps].w];
    if (active && W.live && !*W.live) active = false;   // a batch system that has stopped
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = 0.f;
    if (active) {
        for (int first = 0; first < sp.z; first += kGroupChunk) {
            const int cnt = min(kGroupChunk, sp.z - first);
            __syncwarp();
            for (int i = lane; i < cnt * 8; i += 32) {
                const int p = i >> 3, k = i & 7;
                const int64_t pos = (int64_t)sp.y + first + p;
                float4 v = reinterpret_cast<const float4*>(W.wtab + pos * 32)[k];
                if (k < 4) {
                    const float al = W.asort[pos];
                    v.x *= al; v.y *= al; v.z *= al; v.w *= al;
                    reinterpret_cast<float4*>(sx[warp][p])[k] = v;
                } else {
                    reinterpret_cast<float4*>(sy[warp][p])[k - 4] = v;
                }
            }
            __syncwarp();
            if (a < R)
                for (int p = 0; p < cnt; p++) {
                    const float wa = sx[warp][p][a];
                    const float4 y0 = *reinterpret_cast<const float4*>(&sy[warp][p][8 * h]);
                    const float4 y1 = *reinterpret_cast<const float4*>(&sy[warp][p][8 * h + 4]);
                    acc[0] = fmaf(wa, y0.x, acc[0]); acc[1] = fmaf(wa, y0.y, acc[1]);
                    acc[2] = fmaf(wa, y0.z, acc[2]); acc[3] = fmaf(wa, y0.w, acc[3]);
                    acc[4] = fmaf(wa, y1.x, acc[4]); acc[5] = fmaf(wa, y1.y, acc[5]);
                    acc[6] = fmaf(wa, y1.z, acc[6]); acc[7] = fmaf(wa, y1.w, acc[7]);
                }
        }
    }
    if (a < 16)
#pragma unroll
        for (int k = 0; k < 8; k++) red[warp][a][8 * h + k] = acc[k];
    if (lane == 0) {
        key[warp][0] = active ? sp.x : -1;
        key[warp][1] = active ? sp.w : -1;
    }
    __syncthreads();
    const bool leader = active && (warp == 0 || key[warp - 1][0] != sp.x || key[warp - 1][1] != sp.w);
    if (!leader) return;
    int last = warp;
    while (last + 1 < kGroupWarps && key[last + 1][0] == sp.x && key[last + 1][1] == sp.w) last++;
    float* __restrict__ grid = static_cast<float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int by = sp.x % nb, bx = sp.x / nb;
    if (a < R) {
        const int ga = wrap_idx(Tb * bx - m + a, nos);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int c = 8 * h + k;
            float v = 0.f;
            for (int w2 = warp; w2 <= last; w2++) v += red[w2][a][c];
            if (c < R) atomicAdd(&grid[ga * nos + wrap_idx(Tb * by - m + c, nos)], v);
        }
    }
}

// 2-D gather: one thread per node.
template <int R>
__global__ void __launch_bounds__(128) k_gather2_f32(const int4* __restrict__ sub, const DenseWin* __restrict__ descs,
                                                     int m) {
    static_assert(R <= kPitch, "region up to 16");
    __shared__ __align__(16) float reg[R * kPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const float* __restrict__ h = static_cast<const float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int by = sp.x % nb, bx = sp.x / nb;
    for (int i = threadIdx.x; i < R * kPitch; i += blockDim.x) {
        const int a = i / kPitch, c = i % kPitch;
        reg[i] = (c < R) ? h[wrap_idx(Tb * bx - m + a, nos) * nos + wrap_idx(Tb * by - m + c, nos)] : 0.f;
    }
    __syncthreads();
    float* __restrict__ out = static_cast<float*>(W.out);
    for (int q = threadIdx.x; q < sp.z; q += blockDim.x) {
        const int64_t pos = (int64_t)sp.y + q;
        const float4* wp = reinterpret_cast<const float4*>(W.wtab + pos * 32);
        float wx[16], wy[16];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float4 x = wp[k], y = wp[4 + k];
            wx[4 * k] = x.x; wx[4 * k + 1] = x.y; wx[4 * k + 2] = x.z; wx[4 * k + 3] = x.w;
            wy[4 * k] = y.x; wy[4 * k + 1] = y.y; wy[4 * k + 2] = y.z; wy[4 * k + 3] = y.w;
        }
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < R; a++) {
            float s = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < (R + 3) / 4; c4++) {
                const float4 v = *reinterpret_cast<const float4*>(&reg[a * kPitch + 4 * c4]);
                const float hv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (4 * c4 + e < R) s = fmaf(wy[4 * c4 + e], hv[e], s);
            }
            acc = fmaf(wx[a], s, acc);
        }
        out[W.perm[pos]] = acc;
    }
}

// 1-D spread: as the 2-D one, lane a < R of each warp keeps cell a of its
// sub-problem's region; warps sharing a bin add up before the grid atomics.
template <int R>
__global__ void __launch_bounds__(32 * kGroupWarps) k_spread1_f32(const int4* __restrict__ sub,
                                                                  const DenseWin* __restrict__ descs, int m,
                                                                  int nsub) {
    static_assert(R <= kPitch, "region up to 16");
    __shared__ __align__(16) float sx[kGroupWarps][kGroupChunk][kPitch];
    __shared__ float red[kGroupWarps][32];
    __shared__ int key[kGroupWarps][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int si = blockIdx.x * kGroupWarps + warp;
    int4 sp = make_int4(0, 0, 0, 0);
    bool active = si < nsub;
    if (active) sp = sub[si];
    const DenseWin W = descs[active ? sp.w : sub[blockIdx.x * kGroupWarps].w];
    if (active && W.live && !*W.live) active = false;   // a batch system that has stopped
    float acc = 0.f;
    if (active) {
        for (int first = 0; first < sp.z; first += kGroupChunk) {
            const int cnt = min(kGroupChunk, sp.z - first);
            __syncwarp();
            for (int i = lane; i < cnt * 4; i += 32) {
                const int p = i >> 2, k = i & 3;
                const int64_t pos = (int64_t)sp.y + first + p;
                float4 v = reinterpret_cast<const float4*>(W.wtab + pos * 16)[k];
                const float al = W.asort[pos];
                v.x *= al; v.y *= al; v.z *= al; v.w *= al;
                reinterpret_cast<float4*>(sx[warp][p])[k] = v;
            }
            __syncwarp();
            if (lane < R)
                for (int p = 0; p < cnt; p++) acc += sx[warp][p][lane];
        }
    }
    red[warp][lane] = acc;
    if (lane == 0) {
        key[warp][0] = active ? sp.x : -1;
        key[warp][1] = active ? sp.w : -1;
    }
    __syncthreads();
    const bool leader = active && (warp == 0 || key[warp - 1][0] != sp.x || key[warp - 1][1] != sp.w);
    if (!leader) return;
    int last = warp;
    while (last + 1 < kGroupWarps && key[last + 1][0] == sp.x && key[last + 1][1] == sp.w) last++;
    if (lane < R) {
        float v = 0.f;
        for (int w2 = warp; w2 <= last; w2++) v += red[w2][lane];
        float* __restrict__ grid = static_cast<float*>(W.grid);
        atomicAdd(&grid[wrap_idx(W.Tb * sp.x - m + lane, W.nos)], v);
    }
}

// 1-D gather: one thread per node.
template <int R>
__global__ void __launch_bounds__(128) k_gather1_f32(const int4* __restrict__ sub, const DenseWin* __restrict__ descs,
                                                     int m) {
    static_assert(R <= kPitch, "region up to 16");
    __shared__ __align__(16) float reg[kPitch];
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const float* __restrict__ h = static_cast<const float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb;
    const int bx = sp.x;
    if (threadIdx.x < kPitch) reg[threadIdx.x] = (threadIdx.x < R) ? h[wrap_idx(Tb * bx - m + threadIdx.x, nos)] : 0.f;
    __syncthreads();
    float* __restrict__ out = static_cast<float*>(W.out);
    for (int q = threadIdx.x; q < sp.z; q += blockDim.x) {
        const int64_t pos = (int64_t)sp.y + q;
        const float4* wp = reinterpret_cast<const float4*>(W.wtab + pos * 16);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float4 x = wp[k];
            const float4 v = *reinterpret_cast<const float4*>(&reg[4 * k]);
            acc = fmaf(x.x, v.x, fmaf(x.y, v.y, fmaf(x.z, v.z, fmaf(x.w, v.w, acc))));
        }
        out[W.perm[pos]] = acc;
    }
}

template <typename T>
static const T* frac_of3(const PointSet& ps);
template <>
const double* frac_of3<double>(const PointSet& ps) { return ps.frac64; }
template <>
const float* frac_of3<float>(const PointSet& ps) { return ps.frac32; }

template <typename T, int R>
static void launch_spread(anova_plan* plan, const int4* sub, int nsub, const DenseWin* descs, const DenseWin& one,
                          const void* alpha, int alpha_double, cudaStream_t st) {
    constexpr int NT = R * (R / 2 + R % 2) * 2;
    k_spread3_dense<T, R><<<nsub, NT, 0, st>>>(sub, descs, one, alpha, alpha_double, plan->m, (T)plan->b,
                                               (T)plan->psi_norm, plan->psi_poly);
}

template <typename T, int R>
static void launch_gather(anova_plan* plan, const int4* sub, int nsub, const DenseWin* descs, const DenseWin& one,
                          cudaStream_t st) {
    k_gather3_dense<T, R><<<nsub, kGatherThreads, 0, st>>>(sub, descs, one, plan->m, (T)plan->b,
                                                           (T)plan->psi_norm, plan->psi_poly);
}

template <typename T>
static anova_status spread_dispatch(anova_plan* plan, int R, const int4* sub, int nsub, const DenseWin* descs,
                                    const DenseWin& one, const void* alpha, int alpha_double, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    switch (R) {
        case 4: launch_spread<T, 4>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 6: launch_spread<T, 6>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 8: launch_spread<T, 8>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 10: launch_spread<T, 10>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 12: launch_spread<T, 12>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 14: launch_spread<T, 14>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        case 16: launch_spread<T, 16>(plan, sub, nsub, descs, one, alpha, alpha_double, st); break;
        default: set_error("dense 3-D spread: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

template <typename T>
static anova_status gather_dispatch(anova_plan* plan, int R, const int4* sub, int nsub, const DenseWin* descs,
                                    const DenseWin& one, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    switch (R) {
        case 4: launch_gather<T, 4>(plan, sub, nsub, descs, one, st); break;
        case 6: launch_gather<T, 6>(plan, sub, nsub, descs, one, st); break;
        case 8: launch_gather<T, 8>(plan, sub, nsub, descs, one, st); break;
        case 10: launch_gather<T, 10>(plan, sub, nsub, descs, one, st); break;
        case 12: launch_gather<T, 12>(plan, sub, nsub, descs, one, st); break;
        case 14: launch_gather<T, 14>(plan, sub, nsub, descs, one, st); break;
        case 16: launch_gather<T, 16>(plan, sub, nsub, descs, one, st); break;
        default: set_error("dense 3-D gather: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

static DenseWin single_desc(const WindowPlan& w, const PointSet& ps, const void* frac, void* grid, void* out) {
    DenseWin d;
    d.perm = ps.perm;
    d.cell = ps.cell;
    d.frac = frac;
    d.wtab = nullptr;
    d.wtap = (&ps == &w.X) ? w.wtap64 : nullptr;   // the tap table describes the plan's own nodes only
    d.asort = nullptr;
    d.grid = grid;
    d.out = out;
    d.N = ps.N;
    d.nos = w.nos;
    d.Tb = w.T;
    d.nb = w.nb;
    d.pad = 0;
    return d;
}

// one window, any node set (used by prediction and the debug entry point)
template <typename T>
anova_status spread3_dense(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const void* alpha,
                           int alpha_double, T* grid, cudaStream_t st) {
    const DenseWin one = single_desc(w, ps, frac_of3<T>(ps), grid, nullptr);
    return spread_dispatch<T>(plan, w.R, ps.sub, ps.nsub, nullptr, one, alpha, alpha_double, st);
}

template <typename T>
anova_status gather3_dense(anova_plan* plan, const WindowPlan& w, const PointSet& ps, const T* h, T* out,
                           cudaStream_t st) {
    const DenseWin one = single_desc(w, ps, frac_of3<T>(ps), const_cast<T*>(h), out);
    return gather_dispatch<T>(plan, w.R, ps.sub, ps.nsub, nullptr, one, st);
}

// all dense windows of the plan on their training nodes, one launch per region size
// FP32 windows with a weight table and an even region use the packed kernels
static bool table_kernels(const anova_plan* plan, int R) {
    return (plan->precision & ANOVA_FP32) && R % 2 == 0 && R >= 4 && R <= 16;
}

static anova_status spread_table(anova_plan* plan, int R, const int4* sub, int nsub, const DenseWin* descs,
                                 const void* alpha, int alpha_double, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    if (plan->spread_tc5 && tc5_supported(R, plan->m))
        return spread3_tc5(R, plan->m, sub, nsub, descs, plan->psi_host.data(), plan->sm_count, alpha, alpha_double,
                           st);
    if (plan->spread_tc && plan->spread_f16 && alpha)
        return spread3_f16(R, plan->m, sub, nsub, descs, alpha, alpha_double, plan->N, plan->f16_scale,
                           plan->sm_count, st);
    if (plan->spread_tc && plan->spread_pipe) {
        switch (R) {
#define ANOVA_SPREAD_TCP(R_) \
    case R_: k_spread3_tcp<R_><<<nsub, 32 * (R_ / 2), 0, st>>>(sub, descs, plan->m, alpha, alpha_double); ANOVA_CHECK_LAUNCH(); return ANOVA_OK;
            ANOVA_SPREAD_TCP(4) ANOVA_SPREAD_TCP(6) ANOVA_SPREAD_TCP(8) ANOVA_SPREAD_TCP(10) ANOVA_SPREAD_TCP(12)
            ANOVA_SPREAD_TCP(14) ANOVA_SPREAD_TCP(16)
#undef ANOVA_SPREAD_TCP
            default: break;
        }
    }
    if (plan->spread_tc) {
        switch (R) {
#define ANOVA_SPREAD_TC(R_) \
    case R_: k_spread3_tc<R_><<<nsub, 32 * (R_ / 2), 0, st>>>(sub, descs, plan->m, alpha, alpha_double); ANOVA_CHECK_LAUNCH(); return ANOVA_OK;
            ANOVA_SPREAD_TC(4) ANOVA_SPREAD_TC(6) ANOVA_SPREAD_TC(8) ANOVA_SPREAD_TC(10) ANOVA_SPREAD_TC(12)
            ANOVA_SPREAD_TC(14) ANOVA_SPREAD_TC(16)
#undef ANOVA_SPREAD_TC
            default: break;
        }
    }
    switch (R) {
#define ANOVA_SPREAD_T(R_) \
    case R_: k_spread3_f32<R_><<<nsub, R_ * (R_ / 2) * 2, 0, st>>>(sub, descs, alpha, alpha_double, plan->m); break;
        ANOVA_SPREAD_T(4) ANOVA_SPREAD_T(6) ANOVA_SPREAD_T(8) ANOVA_SPREAD_T(10) ANOVA_SPREAD_T(12)
        ANOVA_SPREAD_T(14) ANOVA_SPREAD_T(16)
#undef ANOVA_SPREAD_T
        default: set_error("dense 3-D spread: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

static anova_status gather_table(anova_plan* plan, int R, const int4* sub, int nsub, const DenseWin* descs,
                                 cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    if (plan->gather_tc5 && tc5_supported(R, plan->m) && tc5_gather_pays(nsub, plan->sm_count))
        return gather3_tc5(R, plan->m, sub, nsub, descs, plan->psi_host.data(), plan->sm_count, st);
    if (plan->gather_tc && plan->gather_umma) return gather3_umma(R, sub, nsub, descs, plan->m, plan->psi_poly, st);
    if (plan->gather_tc) {
        switch (R) {
#define ANOVA_GATHER_TC(R_) \
    case R_: k_gather3_tc<R_><<<nsub, kGatherTcThreads, 0, st>>>(sub, descs, plan->m); ANOVA_CHECK_LAUNCH(); return ANOVA_OK;
            ANOVA_GATHER_TC(4) ANOVA_GATHER_TC(6) ANOVA_GATHER_TC(8) ANOVA_GATHER_TC(10) ANOVA_GATHER_TC(12)
            ANOVA_GATHER_TC(14) ANOVA_GATHER_TC(16)
#undef ANOVA_GATHER_TC
            default: break;
        }
    }
    switch (R) {
#define ANOVA_GATHER_T(R_) \
    case R_: k_gather3_f32<R_><<<nsub, kGather2Threads, 0, st>>>(sub, descs, plan->m); break;
        ANOVA_GATHER_T(4) ANOVA_GATHER_T(6) ANOVA_GATHER_T(8) ANOVA_GATHER_T(10) ANOVA_GATHER_T(12)
        ANOVA_GATHER_T(14) ANOVA_GATHER_T(16)
#undef ANOVA_GATHER_T
        default: set_error("dense 3-D gather: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// FP32 dense kernels over any merged sub-problem list whose descriptors carry
// sorted coefficients (plans and batches alike): one launch per (dims, R) group.
anova_status dense_f32_spread_groups(int m, const int4* sub_base, const DenseWin* descs,
                                     const std::vector<std::array<int, 3>>& groups, cudaStream_t st,
                                     const float* psi_host, int sms, bool tc5_3d) {
    for (const auto& g : groups) {
        const int dA = g[0] / 100, R = g[0] % 100;
        const int4* sub = sub_base + g[1];
        const int nsub = g[2];
        if (nsub == 0) continue;
        if (dA < 3 && psi_host && tc5_supported(R, m)) {
            ANOVA_TRY(dense12_pw(dA, true, R, m, sub, nsub, descs, psi_host, sms, nullptr, 0, st));
            continue;
        }
        switch (dA * 100 + R) {
#define ANOVA_S(R_)                                                                           \
    case 100 + R_: k_spread1_f32<R_><<<(nsub + kGroupWarps - 1) / kGroupWarps, 32 * kGroupWarps, 0, st>>>(sub, descs, m, nsub); break;              \
    case 200 + R_: k_spread2_f32<R_><<<(nsub + kGroupWarps - 1) / kGroupWarps, 32 * kGroupWarps, 0, st>>>(sub, descs, m, nsub); break;              \
    case 300 + R_:                                                                            \
        if (tc5_3d && psi_host && tc5_supported(R_, m)) {                                     \
            ANOVA_TRY(spread3_tc5(R_, m, sub, nsub, descs, psi_host, sms, nullptr, 0, st));   \
            continue;                                                                         \
        }                                                                                     \
        k_spread3_tcp<R_><<<nsub, 32 * (R_ / 2), 0, st>>>(sub, descs, m); break;
            ANOVA_S(4) ANOVA_S(6) ANOVA_S(8) ANOVA_S(10) ANOVA_S(12) ANOVA_S(14) ANOVA_S(16)
#undef ANOVA_S
            default: set_error("dense FP32 spread: unsupported window dimension or region size"); return ANOVA_EINVAL;
        }
        ANOVA_CHECK_LAUNCH();
    }
    return ANOVA_OK;
}

anova_status dense_f32_gather_groups(int m, const float* poly, const int4* sub_base, const DenseWin* descs,
                                     const std::vector<std::array<int, 3>>& groups, cudaStream_t st,
                                     const float* psi_host, int sms) {
    for (const auto& g : groups) {
        const int dA = g[0] / 100, R = g[0] % 100;
        const int4* sub = sub_base + g[1];
        const int nsub = g[2];
        if (nsub == 0) continue;
        if (dA < 3 && psi_host && tc5_supported(R, m)) {
            ANOVA_TRY(dense12_pw(dA, false, R, m, sub, nsub, descs, psi_host, sms, nullptr, 0, st));
            continue;
        }
        switch (dA * 100 + R) {
#define ANOVA_G(R_)                                                                           \
    case 100 + R_: k_gather1_f32<R_><<<nsub, 128, 0, st>>>(sub, descs, m); break;             \
    case 200 + R_: k_gather2_f32<R_><<<nsub, 128, 0, st>>>(sub, descs, m); break;             \
    case 300 + R_:                                                                            \
        if (psi_host && tc5_supported(R_, m) && tc5_gather_pays(nsub, sms))                   \
            ANOVA_TRY(gather3_tc5(R_, m, sub, nsub, descs, psi_host, sms, st));               \
        else ANOVA_TRY(gather3_umma(R_, sub, nsub, descs, m, poly, st));                      \
        break;
            ANOVA_G(4) ANOVA_G(6) ANOVA_G(8) ANOVA_G(10) ANOVA_G(12) ANOVA_G(14) ANOVA_G(16)
#undef ANOVA_G
            default: set_error("dense FP32 gather: unsupported window dimension or region size"); return ANOVA_EINVAL;
        }
        ANOVA_CHECK_LAUNCH();
    }
    return ANOVA_OK;
}

template <typename T>
anova_status dense3_spread_all(anova_plan* plan, const void* alpha, int alpha_double, cudaStream_t st,
                              int* launches, int dims) {
    const int nd = (int)plan->dense_windows.size();
    const DenseWin* descs = plan->dense_desc + (sizeof(T) == 8 ? 0 : nd);
    // the sorted coefficient copies serve the 1-D / 2-D kernels and the packed
    // FP32 3-D ones; the tensor-core 3-D spread gathers through the permutation
    bool need_sort = false;
    for (const auto& g : plan->dense_groups) {
        const int dA = g[0] / 100, R = g[0] % 100;
        const bool ok12 = plan->pw12 && tc5_supported(R, plan->m);
        const bool ok3 = (plan->spread_tc5 && tc5_supported(R, plan->m)) || plan->spread_tc;
        if (dA < 3 ? !ok12 : !ok3) need_sort = true;
    }
    if ((dims & kDenseSort) && sizeof(T) == 4 && plan->dense_asort && need_sort) {
        k_sort_alpha<<<grid_for(plan->N * nd, kThreads, 8 * plan->sm_count), kThreads, 0, st>>>(
            descs, nd, plan->N, alpha, alpha_double);
        ANOVA_CHECK_LAUNCH();
        if (launches) ++*launches;
    }
    for (const auto& g : plan->dense_groups) {
        const int dA = g[0] / 100, R = g[0] % 100;
        const int4* sub = plan->dense_sub + g[1];
        const int nsub = g[2];
        if (!(dims & (dA < 3 ? kDense12 : kDense3))) continue;
        if (launches) ++*launches;
        if (dA < 3) {
            if (sizeof(T) != 4 || !plan->dense_asort) continue;   // FP64: generic kernels per window
            if (plan->pw12 && tc5_supported(R, plan->m)) {
                ANOVA_TRY(dense12_pw(dA, true, R, plan->m, sub, nsub, descs, plan->psi_host.data(), plan->sm_count,
                                     alpha, alpha_double, st));
                continue;
            }
            if (dA == 2) {
                switch (R) {
#define ANOVA_S2(R_) case R_: k_spread2_f32<R_><<<(nsub + kGroupWarps - 1) / kGroupWarps, 32 * kGroupWarps, 0, st>>>(sub, descs, plan->m, nsub); break;
                    ANOVA_S2(4) ANOVA_S2(6) ANOVA_S2(8) ANOVA_S2(10) ANOVA_S2(12) ANOVA_S2(14) ANOVA_S2(16)
#undef ANOVA_S2
                    default: set_error("dense 2-D spread: unsupported region size"); return ANOVA_EINVAL;
                }
            } else {
                switch (R) {
#define ANOVA_S1(R_) case R_: k_spread1_f32<R_><<<(nsub + kGroupWarps - 1) / kGroupWarps, 32 * kGroupWarps, 0, st>>>(sub, descs, plan->m, nsub); break;
                    ANOVA_S1(4) ANOVA_S1(6) ANOVA_S1(8) ANOVA_S1(10) ANOVA_S1(12) ANOVA_S1(14) ANOVA_S1(16)
#undef ANOVA_S1
                    default: set_error("dense 1-D spread: unsupported region size"); return ANOVA_EINVAL;
                }
            }
            ANOVA_CHECK_LAUNCH();
            continue;
        }
        clock_begin(plan, 4, st);
        if (sizeof(T) == 4 && table_kernels(plan, R))
            ANOVA_TRY(spread_table(plan, R, sub, nsub, descs, alpha, alpha_double, st));
        else
            ANOVA_TRY(spread_dispatch<T>(plan, R, sub, nsub, descs, DenseWin(), alpha, alpha_double, st));
        clock_end(plan, 4, 1, st);
    }
    return ANOVA_OK;
}

template <typename T>
anova_status dense3_gather_all(anova_plan* plan, cudaStream_t st, int dims) {
    const int nd = (int)plan->dense_windows.size();
    const DenseWin* descs = plan->dense_desc + (sizeof(T) == 8 ? 0 : nd);
    for (const auto& g : plan->dense_groups) {
        const int dA = g[0] / 100, R = g[0] % 100;
        const int4* sub = plan->dense_sub + g[1];
        const int nsub = g[2];
        if (!(dims & (dA < 3 ? kDense12 : kDense3))) continue;
        if (dA < 3) {
            if (sizeof(T) != 4 || !plan->dense_asort) continue;
            if (plan->pw12 && tc5_supported(R, plan->m)) {
                ANOVA_TRY(dense12_pw(dA, false, R, plan->m, sub, nsub, descs, plan->psi_host.data(), plan->sm_count,
                                     nullptr, 0, st));
                continue;
            }
            if (dA == 2) {
                switch (R) {
#define ANOVA_G2(R_) case R_: k_gather2_f32<R_><<<nsub, 128, 0, st>>>(sub, descs, plan->m); break;
                    ANOVA_G2(4) ANOVA_G2(6) ANOVA_G2(8) ANOVA_G2(10) ANOVA_G2(12) ANOVA_G2(14) ANOVA_G2(16)
#undef ANOVA_G2
                    default: set_error("dense 2-D gather: unsupported region size"); return ANOVA_EINVAL;
                }
            } else {
                switch (R) {
#define ANOVA_G1(R_) case R_: k_gather1_f32<R_><<<nsub, 128, 0, st>>>(sub, descs, plan->m); break;
                    ANOVA_G1(4) ANOVA_G1(6) ANOVA_G1(8) ANOVA_G1(10) ANOVA_G1(12) ANOVA_G1(14) ANOVA_G1(16)
#undef ANOVA_G1
                    default: set_error("dense 1-D gather: unsupported region size"); return ANOVA_EINVAL;
                }
            }
            ANOVA_CHECK_LAUNCH();
            continue;
        }
        clock_begin(plan, 5, st);
        if (sizeof(T) == 4 && table_kernels(plan, R))
            ANOVA_TRY(gather_table(plan, R, sub, nsub, descs, st));
        else
            ANOVA_TRY(gather_dispatch<T>(plan, R, sub, nsub, descs, DenseWin(), st));
        clock_end(plan, 5, 1, st);
    }
    return ANOVA_OK;
}

// region size and sub-problem count of the plan's 3-D dense windows (0: none)
static int region3(const anova_plan* plan, int* nsub = nullptr) {
    for (const auto& g : plan->dense_groups)
        if (g[0] / 100 == 3) {
            if (nsub) *nsub = g[2];
            return g[0] % 100;
        }
    return 0;
}

// kernel names of the FP32 3-D spread and gather the plan launches ("<R>" = region size)
static const char* spread3_name(const anova_plan* plan) {
    if (plan->spread_tc5 && tc5_supported(region3(plan), plan->m)) return "k_spread3_tc5<R>";
    if (plan->spread_tc && plan->spread_f16) return "k_spread3_tch<R>";
    if (plan->spread_tc && plan->spread_pipe) return "k_spread3_tcp<R>";
    return plan->spread_tc ? "k_spread3_tc<R>" : "k_spread3_f32<R>";
}
static const char* gather3_name(const anova_plan* plan) {
    int n3 = 0;
    const int R3 = region3(plan, &n3);
    if (plan->gather_tc5 && tc5_supported(R3, plan->m) && tc5_gather_pays(n3, plan->sm_count)) return "k_gather3_tc5<R>";
    if (plan->gather_tc && plan->gather_umma) return "k_gather3_umma<R>";
    return plan->gather_tc ? "k_gather3_tc<R>" : "k_gather3_f32<R>";
}

template anova_status dense3_spread_all<float>(anova_plan*, const void*, int, cudaStream_t, int*, int);
template anova_status dense3_spread_all<double>(anova_plan*, const void*, int, cudaStream_t, int*, int);
template anova_status dense3_gather_all<float>(anova_plan*, cudaStream_t, int);
template anova_status dense3_gather_all<double>(anova_plan*, cudaStream_t, int);
template anova_status spread3_dense<float>(anova_plan*, const WindowPlan&, const PointSet&, const void*, int,
                                           float*, cudaStream_t);
template anova_status spread3_dense<double>(anova_plan*, const WindowPlan&, const PointSet&, const void*, int,
                                            double*, cudaStream_t);
template anova_status gather3_dense<float>(anova_plan*, const WindowPlan&, const PointSet&, const float*, float*,
                                           cudaStream_t);
template anova_status gather3_dense<double>(anova_plan*, const WindowPlan&, const PointSet&, const double*,
                                            double*, cudaStream_t);

}  // namespace anova

extern "C" anova_status anova_plan_dense3_kernels(const anova_plan* plan, const char** spread, const char** gather) {
    if (!plan || !spread || !gather) {
        anova::set_error("anova_plan_dense3_kernels: NULL argument");
        return ANOVA_EINVAL;
    }
    *spread = anova::spread3_name(plan);
    *gather = anova::gather3_name(plan);
    return ANOVA_OK;
}
