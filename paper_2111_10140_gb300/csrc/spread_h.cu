// spread_h.cu -- the FP32 3-D spread (the window step of the adjoint NFFT,
// Eq. adjnfft, in the fast summation of Sec. 4.2, Eq. fastsum) for every 3-D
// window of a plan in one launch, with the bin's contraction
//   C[(a,b)][c] = sum_p (wx_p[a] wy_p[b]) (alpha_p wz_p[c] / s)
// on mma.sync m16n8k16 with FP16 operands (M = b, N = c, K = 16 nodes per
// instruction: twice the nodes of the TF32 m16n8k8 form for the same number
// of tensor-core instructions).
//
// Precision.  Every operand lies in [-1, 1]: the window weights are at most
// psi(0) = 1, and the coefficients are divided by s = max_i |alpha_i| (one
// reduction over the vector before the launch; the region is multiplied by s
// when it is added to the grid).  Each operand x is split into its FP16
// rounding h and the FP16 rounding of x - h; h*h + h*l + l*h accumulate in
// FP32.  A product a*b of operands of at least 2^-2 (normal FP16 tails) is
// kept to 3 * 2^-22 of itself (the dropped l*l and the tails' roundings);
// below that FP16's subnormal spacing adds at most 2^-24 (|a| + |b|), an
// absolute error against operands of at most 1.  The result meets the FP32
// bar of the product (1e-5 relative); terms that are tiny against the bin's
// largest lose relative, not absolute, accuracy.
//
// Layout and pipeline as the TF32 form (k_spread3_tcp): one block per
// sub-problem, warp w owns the M-tiles a = 2w, 2w+1 and both N-tiles; chunks
// of 64 nodes, the next chunk's weight-table rows and coefficients copied by
// cp.async into the other of two buffers while the current chunk's MMAs run.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "psi.cuh"

namespace anova {

namespace {

constexpr int kHChunk = 64;      // nodes staged at once (a multiple of the MMA's K = 16)
constexpr int kHPitch = 52;      // floats per staged row: rows 2t apart fall in distinct bank groups
constexpr int kHBPitch = 36;     // 32-bit words (node pairs) per B row: c rows 4 banks apart

__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// (x0, x1) as FP16 heads and FP16 tails, packed in pairs (x0 in the low half)
__device__ __forceinline__ void f16_split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void mma_f16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// bits of max_i |alpha_i| (non-negative floats order as unsigned integers); *out zeroed before
template <typename T>
__global__ void __launch_bounds__(kThreads) k_absmax(const T* __restrict__ alpha, int64_t N, unsigned* __restrict__ out) {
    __shared__ unsigned sh[kThreads / 32];
    unsigned m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf((float)alpha[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(out, m);
    }
}

template <int R>
__global__ void __launch_bounds__(32 * (R / 2), (R <= 14 ? 5 : 4))
k_spread3_tch(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m, const void* __restrict__ alpha,
              int alpha_double, const unsigned* __restrict__ scale_bits) {
    static_assert(R <= 16 && R % 2 == 0, "even region up to 16");
    constexpr int NW = R / 2;
    constexpr int NT = 32 * NW;
    __shared__ __align__(16) float raw[2][kHChunk][kHPitch];        // x weights 0..15, y 16..31, z 32..47
    __shared__ __align__(16) double sal[2][kHChunk];                // coefficients as copied (FP32 or FP64)
    __shared__ __align__(16) uint32_t sbh[16][kHBPitch];            // B = alpha wz / s: FP16 heads, node pairs
    __shared__ __align__(16) uint32_t sbl[16][kHBPitch];            // and tails
    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    float* __restrict__ grid = static_cast<float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const bool dbl = alpha_double != 0;
    const float s = __uint_as_float(*scale_bits);
    const float inv = s > 0.f ? 1.f / s : 0.f;
    auto stage = [&](int b, int first, int32_t pm) {
        const int cnt = min(kHChunk, sp.z - first);
        for (int i = tid; i < cnt * 12; i += NT) {
            const int p = i / 12, k = i % 12;
            cp16(&raw[b][p][4 * k], W.wtab + ((int64_t)sp.y + first + p) * 48 + 4 * k);
        }
        if (tid < cnt) {
            if (dbl) cp8(&sal[b][tid], static_cast<const double*>(alpha) + pm);
            else cp4(&sal[b][tid], static_cast<const float*>(alpha) + pm);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto perm_of = [&](int first) -> int32_t {
        return (first + tid < sp.z && tid < kHChunk) ? W.perm[(int64_t)sp.y + first + tid] : 0;
    };
    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.f;
    stage(0, 0, perm_of(0));
    int32_t pnext = perm_of(kHChunk);
    int b = 0;
    for (int first = 0; first < sp.z; first += kHChunk, b ^= 1) {
        const int cnt = min(kHChunk, sp.z - first);
        const int cnt16 = (cnt + 15) & ~15;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();          // chunk `first` is in buffer b; the MMAs of the previous chunk are done
        if (first + kHChunk < sp.z) {
            stage(b ^ 1, first + kHChunk, pnext);
            pnext = perm_of(first + 2 * kHChunk);
        }
        // x and y rows of the padding nodes (cnt .. cnt16) are zero: the MMAs read them
        for (int i = tid; i < (cnt16 - cnt) * 32; i += NT) raw[b][cnt + (i >> 5)][i & 31] = 0.f;
        // B: node pairs (2q, 2q + 1) of column c
        for (int i = tid; i < 16 * (cnt16 / 2); i += NT) {
            const int c = i & 15, q = i >> 4, p0 = 2 * q, p1 = p0 + 1;
            float v0 = 0.f, v1 = 0.f;
            if (p0 < cnt) {
                const float al = dbl ? (float)sal[b][p0] : reinterpret_cast<const float*>(&sal[b][p0])[0];
                v0 = al * inv * raw[b][p0][32 + c];
            }
            if (p1 < cnt) {
                const float al = dbl ? (float)sal[b][p1] : reinterpret_cast<const float*>(&sal[b][p1])[0];
                v1 = al * inv * raw[b][p1][32 + c];
            }
            f16_split(v0, v1, sbh[c][q], sbl[c][q]);
        }
        __syncthreads();
        for (int p0 = 0; p0 < cnt16; p0 += 16) {
            const int n0 = p0 + 2 * t, n1 = n0 + 1, n2 = n0 + 8, n3 = n0 + 9;
            const float y00 = raw[b][n0][16 + g], y01 = raw[b][n1][16 + g];
            const float y10 = raw[b][n0][24 + g], y11 = raw[b][n1][24 + g];
            const float y20 = raw[b][n2][16 + g], y21 = raw[b][n3][16 + g];
            const float y30 = raw[b][n2][24 + g], y31 = raw[b][n3][24 + g];
            const int q0 = (p0 >> 1) + t;
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                bh[nt][0] = sbh[8 * nt + g][q0];
                bh[nt][1] = sbh[8 * nt + g][q0 + 4];
                bl[nt][0] = sbl[8 * nt + g][q0];
                bl[nt][1] = sbl[8 * nt + g][q0 + 4];
            }
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int a = 2 * warp + i;
                const float x0 = raw[b][n0][a], x1 = raw[b][n1][a], x2 = raw[b][n2][a], x3 = raw[b][n3][a];
                uint32_t ah[4], alo[4];
                f16_split(x0 * y00, x1 * y01, ah[0], alo[0]);   // row b = g, nodes 2t, 2t + 1
                f16_split(x0 * y10, x1 * y11, ah[1], alo[1]);   // row g + 8
                f16_split(x2 * y20, x3 * y21, ah[2], alo[2]);   // row g, nodes 2t + 8, 2t + 9
                f16_split(x2 * y30, x3 * y31, ah[3], alo[3]);   // row g + 8
#pragma unroll
                for (int nt = 0; nt < 2; nt++) {
                    mma_f16(acc[i][nt], ah, bh[nt][0], bh[nt][1]);
                    mma_f16(acc[i][nt], ah, bl[nt][0], bl[nt][1]);
                    mma_f16(acc[i][nt], alo, bh[nt][0], bh[nt][1]);
                }
            }
        }
    }
    // the region, times s, into the grid (pairs of cells along c as one 8-byte atomic)
    const bool vec_ok = (reinterpret_cast<uintptr_t>(grid) & 7) == 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int a = 2 * warp + i;
        const int ga = wrap_cell(Tb * bx - m + a, nos);
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int bb = g + 8 * h;
                const int c = 8 * nt + 2 * t;
                if (bb < R && c < R) {
                    const int row = (ga * nos + wrap_cell(Tb * by - m + bb, nos)) * nos;
                    const int gc = wrap_cell(Tb * bz - m + c, nos);
                    const float v0 = acc[i][nt][2 * h] * s, v1 = acc[i][nt][2 * h + 1] * s;
                    if (vec_ok && (gc & 1) == 0 && gc + 1 < nos) {
                        atomicAdd(reinterpret_cast<float2*>(&grid[row + gc]), make_float2(v0, v1));
                    } else {
                        atomicAdd(&grid[row + gc], v0);
                        atomicAdd(&grid[row + wrap_cell(Tb * bz - m + c + 1, nos)], v1);
                    }
                }
            }
    }
}

}  // namespace

// The plan's 3-D spread of one region size on the FP16-split kernel; alpha
// (FP32 or FP64, the caller's vector read through each window's permutation)
// must be given.  scale: a device word of the plan (max |alpha|, recomputed here).
anova_status spread3_f16(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const void* alpha,
                         int alpha_double, int64_t N, unsigned* scale, int sms, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    if (!alpha || !scale) {
        set_error("FP16-split spread: needs the coefficient vector and the plan's scale word");
        return ANOVA_EINVAL;
    }
    ANOVA_CUDA_TRY(cudaMemsetAsync(scale, 0, sizeof(unsigned), st));
    if (alpha_double)
        k_absmax<double><<<grid_for(N, kThreads, 2 * sms), kThreads, 0, st>>>(static_cast<const double*>(alpha), N,
                                                                            scale);
    else
        k_absmax<float><<<grid_for(N, kThreads, 2 * sms), kThreads, 0, st>>>(static_cast<const float*>(alpha), N,
                                                                           scale);
    switch (R) {
#define ANOVA_SPREAD_H(R_) \
    case R_: k_spread3_tch<R_><<<nsub, 32 * (R_ / 2), 0, st>>>(sub, descs, m, alpha, alpha_double, scale); break;
        ANOVA_SPREAD_H(4) ANOVA_SPREAD_H(6) ANOVA_SPREAD_H(8) ANOVA_SPREAD_H(10) ANOVA_SPREAD_H(12)
        ANOVA_SPREAD_H(14) ANOVA_SPREAD_H(16)
#undef ANOVA_SPREAD_H
        default: set_error("FP16-split spread: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

}  // namespace anova
