// dense12.cu -- FP32 spreading and gathering for 1-D and 2-D windows (the
// window steps of the adjoint NFFT, Eq. adjnfft, and of the NFFT, Eq. nfft, in
// the fast summation of Sec. 4.2) on the dense bin regions, with the window
// weights evaluated from each node's cell and offset (psi.cuh) instead of read
// from a per-node table.
//
// Persistent blocks: block k takes a contiguous range of the merged
// sub-problem list (bin, first node, count <= 256, window), with each node's
// data loaded one sub-problem ahead of its use (NodeAhead).  Consecutive
// sub-problems of one bin share the bin's region (R = Tb + 2m cells per axis
// starting at bin*Tb - m):
//   gather  the region is staged in shared memory once per bin; one thread per
//           node forms wx, wy and s = sum_a wx[a] sum_b wy[b] h[a][b];
//   spread  the block's warps split a sub-problem's nodes; each warp keeps the
//           region in registers over up to kFlushSubs sub-problems of the bin,
//           then the block adds its warps' regions to the grid (one set of
//           atomics per kFlushSubs sub-problems instead of one per sub-problem).
// The spread reads each node's coefficient through the node permutation from
// the caller's vector (or a batch instance's sorted copy).
#include <cuda_runtime.h>

#include "common.cuh"
#include "psi.cuh"

namespace anova {

constexpr int k12Threads = 256;          // one thread per node of a sub-problem (kSubChunk)
constexpr int k12Warps = k12Threads / 32;
// the spreads add their register regions to the grid at least every kFlushSubs
// sub-problems, which bounds every FP32 running sum to kFlushSubs x 32 terms
constexpr int kFlushSubs = 4;
static_assert(kSubChunk == k12Threads, "one thread per node of a sub-problem");

__device__ __forceinline__ float coef_of(const DenseWin& W, const void* alpha, int alpha_double, int64_t pos) {
    if (!alpha) return W.asort[pos];
    const int32_t i = W.perm[pos];
    return alpha_double ? (float)static_cast<const double*>(alpha)[i] : static_cast<const float*>(alpha)[i];
}

// A node's data, loaded one sub-problem ahead of its use: while a block computes
// sub-problem q, the loads of q + 1 are in flight (and the sub-problem entry of
// q + 2, which those loads need next time).  idx is the node's original index
// (its entry of the window's permutation); al the coefficient where it is read
// from a sorted copy (no permutation).
template <int DA>
struct NodeAhead {
    float f[DA];
    int c[DA];
    int32_t idx;
    float al;
};

template <int DA>
__device__ __forceinline__ void node_ahead(const DenseWin* __restrict__ descs, const int4& sp, int t, bool sorted_coef,
                                           NodeAhead<DA>& nd) {
    const DenseWin& W = descs[sp.w];
    if (t < sp.z) {
        const int64_t pos = (int64_t)sp.y + t, Nn = W.N;
        const float* __restrict__ fr = static_cast<const float*>(W.frac);
#pragma unroll
        for (int d = 0; d < DA; d++) {
            nd.f[d] = fr[d * Nn + pos];
            nd.c[d] = W.cell[d * Nn + pos];
        }
        if (sorted_coef) nd.al = W.asort[pos];
        else nd.idx = W.perm[pos];
    }
}

__device__ __forceinline__ float coef_ahead(const void* alpha, int alpha_double, int32_t idx, float sorted) {
    if (!alpha) return sorted;
    return alpha_double ? (float)static_cast<const double*>(alpha)[idx] : static_cast<const float*>(alpha)[idx];
}

__device__ __forceinline__ int4 sub_at(const int4* __restrict__ sub, int q, int hi) {
    return q < hi ? sub[q] : make_int4(0, 0, 0, 0);
}

// --------------------------------------------------------------- 2-D gather
template <int R, int M>
__global__ void __launch_bounds__(k12Threads, 5)
k_gather2_pw(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
             const __grid_constant__ PsiCoef<M> P) {
    constexpr int TB = R - 2 * M;
    __shared__ __align__(16) float reg[16 * 16];       // region rows a (x), columns b (y), zero padded
    const int lo = (int)((int64_t)nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)nsub * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x;
    int cw = -1, cbin = -1;
    int4 spA = sub_at(sub, lo, hi), spB = sub_at(sub, lo + 1, hi), spC;
    NodeAhead<2> ndA = {}, ndB = {};
    if (lo < hi) node_ahead<2>(descs, spA, tid, false, ndA);
    for (int q = lo; q < hi; q++, spA = spB, spB = spC, ndA = ndB) {
        spC = sub_at(sub, q + 2, hi);
        if (q + 1 < hi) node_ahead<2>(descs, spB, tid, false, ndB);
        const int4 sp = spA;
        const DenseWin& W = descs[sp.w];
        if (W.live && !*W.live) continue;              // a batch system that has stopped
        const int nb = W.nb, by = sp.x % nb, bx = sp.x / nb;
        if (sp.w != cw || sp.x != cbin) {
            __syncthreads();
            const float* __restrict__ h = static_cast<const float*>(W.grid);
            const int nos = W.nos, a = tid >> 4, b = tid & 15;
            reg[tid] = (a < R && b < R) ? h[wrap_cell(TB * bx - M + a, nos) * nos + wrap_cell(TB * by - M + b, nos)]
                                        : 0.f;
            __syncthreads();
            cw = sp.w;
            cbin = sp.x;
        }
        if (tid < sp.z) {
            float t[2 * M], wx[16], wy[16];
            psi_taps<M>(P, ndA.f[0], t);
            place_taps<R, M>(t, ndA.c[0] - TB * bx, wx);
            psi_taps<M>(P, ndA.f[1], t);
            place_taps<R, M>(t, ndA.c[1] - TB * by, wy);
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < R; a++) {
                float e0 = 0.f, e1 = 0.f;
#pragma unroll
                for (int b4 = 0; b4 < (R + 3) / 4; b4++) {
                    const float4 v = reinterpret_cast<const float4*>(reg)[a * 4 + b4];
                    const float hv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        if (4 * b4 + e >= R) continue;
                        if (e & 1) e1 = fmaf(wy[4 * b4 + e], hv[e], e1);
                        else e0 = fmaf(wy[4 * b4 + e], hv[e], e0);
                    }
                }
                s = fmaf(wx[a], e0 + e1, s);
            }
            static_cast<float*>(W.out)[ndA.idx] = s;
        }
    }
}

// --------------------------------------------------------------- 1-D gather
template <int R, int M>
__global__ void __launch_bounds__(k12Threads)
k_gather1_pw(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
             const __grid_constant__ PsiCoef<M> P) {
    constexpr int TB = R - 2 * M;
    __shared__ __align__(16) float reg[16];
    const int lo = (int)((int64_t)nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)nsub * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x;
    int cw = -1, cbin = -1;
    int4 spA = sub_at(sub, lo, hi), spB = sub_at(sub, lo + 1, hi), spC;
    NodeAhead<1> ndA = {}, ndB = {};
    if (lo < hi) node_ahead<1>(descs, spA, tid, false, ndA);
    for (int q = lo; q < hi; q++, spA = spB, spB = spC, ndA = ndB) {
        spC = sub_at(sub, q + 2, hi);
        if (q + 1 < hi) node_ahead<1>(descs, spB, tid, false, ndB);
        const int4 sp = spA;
        const DenseWin& W = descs[sp.w];
        if (W.live && !*W.live) continue;
        const int bx = sp.x;
        if (sp.w != cw || sp.x != cbin) {
            __syncthreads();
            if (tid < 16)
                reg[tid] = tid < R ? static_cast<const float*>(W.grid)[wrap_cell(TB * bx - M + tid, W.nos)] : 0.f;
            __syncthreads();
            cw = sp.w;
            cbin = sp.x;
        }
        if (tid < sp.z) {
            float t[2 * M], wx[16];
            psi_taps<M>(P, ndA.f[0], t);
            place_taps<R, M>(t, ndA.c[0] - TB * bx, wx);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int a = 0; a < R; a += 2) {
                s0 = fmaf(wx[a], reg[a], s0);
                if (a + 1 < R) s1 = fmaf(wx[a + 1], reg[a + 1], s1);
            }
            static_cast<float*>(W.out)[ndA.idx] = s0 + s1;
        }
    }
}

// --------------------------------------------------------------- 2-D spread
// Warp w takes nodes 32w .. 32w + 31 of a sub-problem: lane p forms its node's
// alpha wx and wy into the warp's staging rows, then lane (a = lane / 2, h =
// lane mod 2) adds alpha_p wx_p[a] wy_p[8h .. 8h + 7] over the 32 nodes.
template <int R, int M>
__global__ void __launch_bounds__(k12Threads)
k_spread2_pw(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
             const __grid_constant__ PsiCoef<M> P, const void* __restrict__ alpha, int alpha_double) {
    constexpr int TB = R - 2 * M;
    constexpr int kPitchS = 20;                         // staging row pitch (conflict-free float4 reads)
    __shared__ __align__(16) float stage[2][k12Warps][32][kPitchS];
    float (*sx)[32][kPitchS] = stage[0];                // alpha wx rows of each warp's nodes
    float (*sy)[32][kPitchS] = stage[1];                // wy rows
    // the flush's per-warp regions reuse the staging rows (between block barriers)
    float (*red)[16][16] = reinterpret_cast<float (*)[16][16]>(&stage[0][0][0][0]);
    const int lo = (int)((int64_t)nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)nsub * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, ra = lane >> 1, rh = lane & 1;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = 0.f;
    int cw = -1, cbin = -1;
    // adds the block's region of bin (cw, cbin) to the grid and clears the accumulators
    auto flush = [&]() {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) {
            red[warp][ra][8 * rh + k] = acc[k];
            acc[k] = 0.f;
        }
        __syncthreads();
        const DenseWin& W = descs[cw];
        const int a = tid >> 4, b = tid & 15;
        if (a < R && b < R) {
            float v = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < k12Warps; w2++) v += red[w2][a][b];
            const int nb = W.nb, by = cbin % nb, bx = cbin / nb, nos = W.nos;
            atomicAdd(&static_cast<float*>(W.grid)[wrap_cell(TB * bx - M + a, nos) * nos + wrap_cell(TB * by - M + b, nos)],
                      v);
        }
        __syncthreads();                                 // the staging rows are free again
    };
    int nacc = 0;                                       // sub-problems in the accumulators
    for (int q = lo; q < hi; q++) {
        const int4 sp = sub[q];
        const DenseWin& W = descs[sp.w];
        if (W.live && !*W.live) continue;
        if (cw >= 0 && (sp.w != cw || sp.x != cbin || nacc == kFlushSubs)) {
            flush();
            nacc = 0;
        }
        cw = sp.w;
        cbin = sp.x;
        nacc++;
        const int nb = W.nb, by = sp.x % nb, bx = sp.x / nb;
        const int p = 32 * warp + lane;
        float wx[16], wy[16];
        if (p < sp.z) {
            const int64_t pos = (int64_t)sp.y + p, Nn = W.N;
            const float* __restrict__ fr = static_cast<const float*>(W.frac);
            const float al = coef_of(W, alpha, alpha_double, pos);
            float t[2 * M];
            psi_taps<M>(P, fr[pos], t);
            place_taps<R, M>(t, W.cell[pos] - TB * bx, wx);
            psi_taps<M>(P, fr[Nn + pos], t);
            place_taps<R, M>(t, W.cell[Nn + pos] - TB * by, wy);
#pragma unroll
            for (int r = 0; r < 16; r++) wx[r] *= al;
        } else {
#pragma unroll
            for (int r = 0; r < 16; r++) wx[r] = wy[r] = 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; k++) {
            reinterpret_cast<float4*>(sx[warp][lane])[k] = make_float4(wx[4 * k], wx[4 * k + 1], wx[4 * k + 2], wx[4 * k + 3]);
            reinterpret_cast<float4*>(sy[warp][lane])[k] = make_float4(wy[4 * k], wy[4 * k + 1], wy[4 * k + 2], wy[4 * k + 3]);
        }
        __syncwarp();
        const int cnt = min(32, sp.z - 32 * warp);
        if (ra < R)
            for (int pp = 0; pp < cnt; pp++) {
                const float wa = sx[warp][pp][ra];
                const float4 y0 = reinterpret_cast<const float4*>(sy[warp][pp])[2 * rh];
                const float4 y1 = reinterpret_cast<const float4*>(sy[warp][pp])[2 * rh + 1];
                acc[0] = fmaf(wa, y0.x, acc[0]); acc[1] = fmaf(wa, y0.y, acc[1]);
                acc[2] = fmaf(wa, y0.z, acc[2]); acc[3] = fmaf(wa, y0.w, acc[3]);
                acc[4] = fmaf(wa, y1.x, acc[4]); acc[5] = fmaf(wa, y1.y, acc[5]);
                acc[6] = fmaf(wa, y1.z, acc[6]); acc[7] = fmaf(wa, y1.w, acc[7]);
            }
    }
    if (cw >= 0) flush();
}

// ------------------------------------------- 2-D spread on tensor cores
// As k_spread2_pw, with each warp's 32-node contribution to its region
// C[a][b] += sum_p (alpha_p wx_p[a]) wy_p[b] run as mma.sync m16n8k8 TF32
// (M = a, N = b in two tiles of 8, K = 8 nodes per step; operands split into
// a TF32 head rounded to nearest and the FP32 residual, head*head + head*tail
// + tail*head in FP32: FP32 accuracy, the dropped tail*tail at most 2^-22 and
// of either sign).  Thread (g = lane / 4, t = lane mod 4)
// holds C[g][8 nt + 2t .. +1] and C[g + 8][8 nt + 2t .. +1] of n-tile nt.
__device__ __forceinline__ void tf32_split2(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32_16x8x8(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int R, int M>
__global__ void __launch_bounds__(k12Threads, 4)
k_spread2_tc(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
             const __grid_constant__ PsiCoef<M> P, const void* __restrict__ alpha, int alpha_double) {
    constexpr int TB = R - 2 * M;
    constexpr int kP = 24;                              // staging row pitch: conflict-free fragment reads
    __shared__ __align__(16) float stage[2][k12Warps][32][kP];
    float (*sx)[32][kP] = stage[0];                     // alpha wx rows of each warp's nodes
    float (*sy)[32][kP] = stage[1];                     // wy rows
    float (*red)[16][16] = reinterpret_cast<float (*)[16][16]>(&stage[0][0][0][0]);
    const int lo = (int)((int64_t)nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)nsub * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float acc[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int k = 0; k < 4; k++) acc[nt][k] = 0.f;
    int cw = -1, cbin = -1;
    auto flush = [&]() {
        __syncthreads();
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            red[warp][g][8 * nt + 2 * t] = acc[nt][0];
            red[warp][g][8 * nt + 2 * t + 1] = acc[nt][1];
            red[warp][g + 8][8 * nt + 2 * t] = acc[nt][2];
            red[warp][g + 8][8 * nt + 2 * t + 1] = acc[nt][3];
#pragma unroll
            for (int k = 0; k < 4; k++) acc[nt][k] = 0.f;
        }
        __syncthreads();
        const DenseWin& W = descs[cw];
        const int a = tid >> 4, b = tid & 15;
        if (a < R && b < R) {
            float v = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < k12Warps; w2++) v += red[w2][a][b];
            const int nb = W.nb, by = cbin % nb, bx = cbin / nb, nos = W.nos;
            atomicAdd(&static_cast<float*>(W.grid)[wrap_cell(TB * bx - M + a, nos) * nos + wrap_cell(TB * by - M + b, nos)],
                      v);
        }
        __syncthreads();                                 // the staging rows are free again
    };
    int nacc = 0;
    int4 spA = sub_at(sub, lo, hi), spB = sub_at(sub, lo + 1, hi), spC;
    NodeAhead<2> ndA = {}, ndB = {};
    if (lo < hi) node_ahead<2>(descs, spA, tid, !alpha, ndA);
    for (int q = lo; q < hi; q++, spA = spB, spB = spC, ndA = ndB) {
        spC = sub_at(sub, q + 2, hi);
        if (q + 1 < hi) node_ahead<2>(descs, spB, tid, !alpha, ndB);
        const int4 sp = spA;
        const DenseWin& W = descs[sp.w];
        if (W.live && !*W.live) continue;
        if (cw >= 0 && (sp.w != cw || sp.x != cbin || nacc == kFlushSubs)) {
            flush();
            nacc = 0;
        }
        cw = sp.w;
        cbin = sp.x;
        nacc++;
        const int nb = W.nb, by = sp.x % nb, bx = sp.x / nb;
        const int p = 32 * warp + lane;
        float wx[16], wy[16];
        if (p < sp.z) {
            const float al = coef_ahead(alpha, alpha_double, ndA.idx, ndA.al);
            float tp[2 * M];
            psi_taps<M>(P, ndA.f[0], tp);
            place_taps<R, M>(tp, ndA.c[0] - TB * bx, wx);
            psi_taps<M>(P, ndA.f[1], tp);
            place_taps<R, M>(tp, ndA.c[1] - TB * by, wy);
#pragma unroll
            for (int r = 0; r < 16; r++) wx[r] *= al;
        } else {
#pragma unroll
            for (int r = 0; r < 16; r++) wx[r] = wy[r] = 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; k++) {
            reinterpret_cast<float4*>(sx[warp][lane])[k] = make_float4(wx[4 * k], wx[4 * k + 1], wx[4 * k + 2], wx[4 * k + 3]);
            reinterpret_cast<float4*>(sy[warp][lane])[k] = make_float4(wy[4 * k], wy[4 * k + 1], wy[4 * k + 2], wy[4 * k + 3]);
        }
        __syncwarp();
        const int cnt = min(32, sp.z - 32 * warp);
        for (int s0 = 0; s0 < cnt; s0 += 8) {
            const int p0 = s0 + t, p1 = s0 + t + 4;
            uint32_t ah[4], al[4];
            tf32_split2(sx[warp][p0][g], ah[0], al[0]);
            tf32_split2(sx[warp][p0][g + 8], ah[1], al[1]);
            tf32_split2(sx[warp][p1][g], ah[2], al[2]);
            tf32_split2(sx[warp][p1][g + 8], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 2; nt++) {
                uint32_t bh0, bl0, bh1, bl1;
                tf32_split2(sy[warp][p0][8 * nt + g], bh0, bl0);
                tf32_split2(sy[warp][p1][8 * nt + g], bh1, bl1);
                mma_tf32_16x8x8(acc[nt], ah, bh0, bh1);
                mma_tf32_16x8x8(acc[nt], ah, bl0, bl1);
                mma_tf32_16x8x8(acc[nt], al, bh0, bh1);
            }
        }
    }
    if (cw >= 0) flush();
}

// --------------------------------------------------------------- 1-D spread
// Every thread keeps the region of the nodes it has seen in registers
// (acc[r] += alpha_p wx_p[r]); per bin the block sums them (warp shuffles, then
// across warps) and adds the region to the grid once.
template <int R, int M>
__global__ void __launch_bounds__(k12Threads)
k_spread1_pw(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
             const __grid_constant__ PsiCoef<M> P, const void* __restrict__ alpha, int alpha_double) {
    constexpr int TB = R - 2 * M;
    __shared__ float red[k12Warps][16];
    const int lo = (int)((int64_t)nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)nsub * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; r++) acc[r] = 0.f;
    int cw = -1, cbin = -1;
    auto flush = [&]() {
#pragma unroll
        for (int r = 0; r < 16; r++) {
            float v = acc[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[r] = 0.f;
            if (lane == 0) red[warp][r] = v;
        }
        __syncthreads();
        if (tid < R) {
            float v = 0.f;
#pragma unroll
            for (int w2 = 0; w2 < k12Warps; w2++) v += red[w2][tid];
            const DenseWin& W = descs[cw];
            atomicAdd(&static_cast<float*>(W.grid)[wrap_cell(TB * cbin - M + tid, W.nos)], v);
        }
        __syncthreads();
    };
    int nacc = 0;                                       // sub-problems in the accumulators
    int4 spA = sub_at(sub, lo, hi), spB = sub_at(sub, lo + 1, hi), spC;
    NodeAhead<1> ndA = {}, ndB = {};
    if (lo < hi) node_ahead<1>(descs, spA, tid, !alpha, ndA);
    for (int q = lo; q < hi; q++, spA = spB, spB = spC, ndA = ndB) {
        spC = sub_at(sub, q + 2, hi);
        if (q + 1 < hi) node_ahead<1>(descs, spB, tid, !alpha, ndB);
        const int4 sp = spA;
        const DenseWin& W = descs[sp.w];
        if (W.live && !*W.live) continue;
        if (cw >= 0 && (sp.w != cw || sp.x != cbin || nacc == kFlushSubs)) {
            flush();
            nacc = 0;
        }
        cw = sp.w;
        cbin = sp.x;
        nacc++;
        if (tid < sp.z) {
            const float al = coef_ahead(alpha, alpha_double, ndA.idx, ndA.al);
            float t[2 * M], w[16];
            psi_taps<M>(P, ndA.f[0], t);
            place_taps<R, M>(t, ndA.c[0] - TB * sp.x, w);
#pragma unroll
            for (int r = 0; r < 16; r++) acc[r] = fmaf(al, w[r], acc[r]);
        }
    }
    if (cw >= 0) flush();
}

// ------------------------------------------------------------------ launches
// blocks of `kernel` resident per SM (looked up once per kernel): the persistent
// kernels launch exactly that many per SM, so their contiguous sub-problem
// ranges run in one wave
template <typename K>
static int resident_blocks(K kernel) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, k12Threads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

template <int R, int M>
static anova_status launch12(int dA, bool spread, const int4* sub, int nsub, const DenseWin* descs,
                             const float* psi_host, int sms, const void* alpha, int alpha_double, cudaStream_t st) {
    const PsiCoef<M> P = psi_coef<M>(psi_host);
    static const int res_s2 = resident_blocks(k_spread2_tc<R, M>), res_g2 = resident_blocks(k_gather2_pw<R, M>);
    static const int res_s1 = resident_blocks(k_spread1_pw<R, M>), res_g1 = resident_blocks(k_gather1_pw<R, M>);
    auto grid_of = [&](int res) { return nsub < res * sms ? nsub : res * sms; };
    if (dA == 2) {
        if (spread)
            k_spread2_tc<R, M><<<grid_of(res_s2), k12Threads, 0, st>>>(sub, nsub, descs, P, alpha, alpha_double);
        else k_gather2_pw<R, M><<<grid_of(res_g2), k12Threads, 0, st>>>(sub, nsub, descs, P);
    } else {
        if (spread)
            k_spread1_pw<R, M><<<grid_of(res_s1), k12Threads, 0, st>>>(sub, nsub, descs, P, alpha, alpha_double);
        else k_gather1_pw<R, M><<<grid_of(res_g1), k12Threads, 0, st>>>(sub, nsub, descs, P);
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// 1-D / 2-D FP32 spread (spread = true) or gather of one group of sub-problems.
// alpha: the caller's coefficients (read through each window's permutation), or
// null for the instances' sorted copies (batches).
anova_status dense12_pw(int dA, bool spread, int R, int m, const int4* sub, int nsub, const DenseWin* descs,
                        const float* psi_host, int sms, const void* alpha, int alpha_double, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
#define ANOVA_P12(R_, M_) \
    if (R == R_ && m == M_) return launch12<R_, M_>(dA, spread, sub, nsub, descs, psi_host, sms, alpha, alpha_double, st);
    ANOVA_P12(10, 4) ANOVA_P12(12, 4) ANOVA_P12(14, 4) ANOVA_P12(16, 4)
    ANOVA_P12(12, 5) ANOVA_P12(14, 5) ANOVA_P12(16, 5)
    ANOVA_P12(14, 6) ANOVA_P12(16, 6)
    ANOVA_P12(16, 7)
#undef ANOVA_P12
    set_error("1-D / 2-D FP32 kernels: unsupported region size or cutoff");
    return ANOVA_EINVAL;
}

}  // namespace anova
