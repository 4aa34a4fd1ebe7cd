// umma.cu -- the FP32 3-D gather (the NFFT step of the fast summation,
// arXiv 2111.10140 Sec. 4.1 Eq. nfft, applied to the convolved grid as in
// Sec. 4.2 Eq. fastsum) on the fifth-generation tensor cores: tcgen05.mma
// with operands in shared memory and the accumulator in tensor memory.
//
// Per sub-problem (one bin, at most 256 nodes, in tiles of 128):
//
//   U[j][(a,b)] = sum_c wz_j[c] h[a][b][c]        (tcgen05.mma, M = 128 nodes,
//                                                   N = R^2 pairs padded to 16,
//                                                   K = 16 z cells)
//   s_j         = sum_(a,b) wx_j[a] wy_j[b] U[j][(a,b)]   (epilogue, CUDA cores)
//
// A (the nodes' z weights) and B (the staged region, row (a,b) holding the R
// cells along z) are split into TF32 heads and tails; head x head, head x
// tail and tail x head accumulate in FP32 in tensor memory, which keeps the
// product at FP32 accuracy.  Operands use the K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes, 128 bytes apart along K and 512 bytes
// apart along M / N; float4 unit u of an operand holds row 8 (u / 32) + u mod 8,
// columns 4 ((u / 8) mod 4) .. +3.  One thread issues the six MMAs of a tile
// and commits them to an mbarrier; every wait on it is bounded and a wait that
// gives up is counted (anova_wait_timeouts).  Thread (warp w, lane l) reads row
// 32 (w mod 4) + l of the accumulator; with 256 threads warps 0-3 and 4-7 take
// half of the columns each.
#include <cuda_runtime.h>

#include "common.cuh"
#include "umma.cuh"

namespace anova {

__device__ unsigned long long g_wait_timeouts = 0;

constexpr int kUmmaThreads = 256;           // 128 (one column group) or 256 (two)
constexpr int kUmmaMinBlocks = 3;           // resident blocks per SM asked of the compiler
constexpr int kUmmaTile = 128;              // nodes per MMA tile (M)
constexpr uint32_t kUmmaCols = 256;         // tensor-memory columns per block (N <= 256)
constexpr size_t kUmmaSmem = 64 * 1024;     // shared memory requested per block at least (three blocks per SM:
                                            // two hold tensor memory, the third stages its operands)
constexpr int kUmmaGroups = kUmmaThreads / 128;   // column groups of the epilogue
// node weights of the gather: evaluated from each node's cell and offset with the plan's
// per-interval FP32 window polynomials (true), or read from the plan's weight table
constexpr bool kGatherPolyW = false;   // measured: 71 us against 45 us with the table (mid workload)
constexpr int kPolyFloats = kGatherPolyW ? 2 * 8 * kPsiStride : 0;   // coefficients for m <= 8
constexpr int kWPitch = 52;                       // staged weight-table rows (floats; conflict-free float4 reads)

// TF32 head and tail of four values (both rounded to nearest)
__device__ __forceinline__ void split4(const float* v, float4& hv, float4& lv) {
    float hh[4], ll[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const uint32_t hi = tf32_rna(v[e]);
        hh[e] = __uint_as_float(hi);
        ll[e] = __uint_as_float(tf32_rna(v[e] - hh[e]));
    }
    hv = make_float4(hh[0], hh[1], hh[2], hh[3]);
    lv = make_float4(ll[0], ll[1], ll[2], ll[3]);
}

template <int R>
__global__ void __launch_bounds__(kUmmaThreads, kUmmaMinBlocks)
k_gather3_umma(const int4* __restrict__ sub, const DenseWin* __restrict__ descs, int m,
               const float* __restrict__ poly) {
    static_assert(R >= 4 && R <= 16 && R % 2 == 0, "even region up to 16");
    constexpr int NP = ((R * R + 15) / 16) * 16;     // MMA N: (a,b) pairs padded to a multiple of 16
    constexpr int NCH = NP / 16;                     // 16-column chunks of the accumulator
    constexpr int PER = (NCH + kUmmaGroups - 1) / kUmmaGroups;   // chunks per column group
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sAh = reinterpret_cast<float*>(sm);       // 128 x 16 z weights: heads
    float* sAl = sAh + kUmmaTile * 16;               //                     tails
    float* sBh = sAl + kUmmaTile * 16;               // NP x 16 region rows: heads
    float* sBl = sBh + NP * 16;                      //                      tails
    float* part = sBl + NP * 16;                     // 128 partial sums of warps 4-7
    float* sP = part + kUmmaTile;                    // window polynomial coefficients
    float* sW = sP + kPolyFloats;                    // 128 x kWPitch: the tile's weight-table rows
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sW + kUmmaTile * kWPitch);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

    const int4 sp = sub[blockIdx.x];
    const DenseWin W = descs[sp.w];
    if (W.live && !*W.live) return;   // a batch system that has stopped
    const float* __restrict__ h = static_cast<const float*>(W.grid);
    const int nos = W.nos, Tb = W.Tb, nb = W.nb;
    const int bz = sp.x % nb, by = (sp.x / nb) % nb, bx = sp.x / (nb * nb);
    const int ox = Tb * bx - m, oy = Tb * by - m, oz = Tb * bz - m;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (kGatherPolyW)
        for (int i = tid; i < 2 * m * kPsiStride + 1; i += kUmmaThreads) sP[i] = poly[i];
    // weight-table rows of the tile starting at node t: asynchronous copies into sW,
    // waited for where they are used (they overlap the region staging and the MMAs)
    auto prefetch = [&](int t) {
        if (kGatherPolyW) return;
        const int rows = min(kUmmaTile, sp.z - t);
        for (int u = tid; u < rows * 12; u += kUmmaThreads) {
            const int node = u / 12, k = u - (u / 12) * 12;
            const float* src = W.wtab + ((int64_t)sp.y + t + node) * 48 + 4 * k;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(sW + node * kWPitch + 4 * k)),
                         "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    prefetch(0);

    // B: row n = (a, b), column c: the region cell (a, b, c), zero beyond R.
    // Unit u (4 consecutive c of one row) goes to float4 u of the operand, so
    // a warp's stores are contiguous: u = (row group, k group, row in group).
#pragma unroll 4
    for (int u = tid; u < NP * 4; u += kUmmaThreads) {
        const int n = (u >> 5) * 8 + (u & 7), c0 = 4 * ((u >> 3) & 3);
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (n < R * R) {
            const int a = n / R, b = n - (n / R) * R;
            int ga = ox + a, gb = oy + b;
            ga += ga < 0 ? nos : (ga >= nos ? -nos : 0);
            gb += gb < 0 ? nos : (gb >= nos ? -nos : 0);
            const float* row = h + ((size_t)ga * nos + gb) * nos;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                int gc = oz + c0 + e;
                gc += gc < 0 ? nos : (gc >= nos ? -nos : 0);
                if (c0 + e < R) v[e] = row[gc];
            }
        }
        float4 hv, lv;
        split4(v, hv, lv);
        reinterpret_cast<float4*>(sBh)[u] = hv;
        reinterpret_cast<float4*>(sBl)[u] = lv;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(kUmmaCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(mbar)), "r"(1));

    constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
                               ((uint32_t)(kUmmaTile >> 4) << 24);
    float* __restrict__ out = static_cast<float*>(W.out);
    uint32_t phase = 0;
    bool ok = true;
    uint32_t taddr = 0;
    for (int t0 = 0; t0 < sp.z && ok; t0 += kUmmaTile) {
        const int rows = min(kUmmaTile, sp.z - t0);
        // Thread (warp w, lane l) owns node row j = 32 (w mod 4) + l of the tile:
        // it loads the node's x and y weights for the epilogue now, and warps
        // 0-3 also its z weights, written as row j of A (zero rows past the
        // bin's nodes) -- one round trip to the weight table per tile.
        const int j = 32 * (warp & 3) + lane;
        const bool valid = j < rows;
        const int64_t pos = (int64_t)sp.y + t0 + (valid ? j : 0);
        float wx[16], wy[16];
        float4 z4[4];
        if (kGatherPolyW) {
            // tap r of axis t: psi(cell - Tb bin + m - r + offset), from the node's cell and offset
            const float* __restrict__ fr = static_cast<const float*>(W.frac);
            const int64_t Nn = W.N;
            const int jx = W.cell[pos] - Tb * bx + m, jy = W.cell[Nn + pos] - Tb * by + m;
            const float fx = fr[pos], fy = fr[Nn + pos];
#pragma unroll
            for (int q = 0; q < 16; q++) {
                wx[q] = q < R ? psi_poly_eval(sP, jx - q, fx, m) : 0.f;
                wy[q] = q < R ? psi_poly_eval(sP, jy - q, fy, m) : 0.f;
            }
            if (warp < 4) {
                const int jz = W.cell[2 * Nn + pos] - Tb * bz + m;
                const float fz = fr[2 * Nn + pos];
                float wz[16];
#pragma unroll
                for (int q = 0; q < 16; q++) wz[q] = (valid && q < R) ? psi_poly_eval(sP, jz - q, fz, m) : 0.f;
#pragma unroll
                for (int kg = 0; kg < 4; kg++) z4[kg] = make_float4(wz[4 * kg], wz[4 * kg + 1], wz[4 * kg + 2], wz[4 * kg + 3]);
            }
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            const float4* wr4 = reinterpret_cast<const float4*>(sW + j * kWPitch);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 x4 = wr4[q];
                const float4 y4 = wr4[4 + q];
                wx[4 * q] = x4.x; wx[4 * q + 1] = x4.y; wx[4 * q + 2] = x4.z; wx[4 * q + 3] = x4.w;
                wy[4 * q] = y4.x; wy[4 * q + 1] = y4.y; wy[4 * q + 2] = y4.z; wy[4 * q + 3] = y4.w;
            }
            if (warp < 4)
#pragma unroll
                for (int kg = 0; kg < 4; kg++) z4[kg] = valid ? wr4[8 + kg] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (warp < 4) {
#pragma unroll
            for (int kg = 0; kg < 4; kg++) {
                const float v[4] = {z4[kg].x, z4[kg].y, z4[kg].z, z4[kg].w};
                float4 hv, lv;
                split4(v, hv, lv);
                const int u = (j >> 3) * 32 + kg * 8 + (j & 7);     // float4 unit of (row j, columns 4 kg ..)
                reinterpret_cast<float4*>(sAh)[u] = hv;
                reinterpret_cast<float4*>(sAl)[u] = lv;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t0 + kUmmaTile < sp.z) prefetch(t0 + kUmmaTile);   // sW is free: every thread holds its weights
        taddr = *tslot;
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint64_t ah = umma_desc(su32(sAh) + ks * 256), al = umma_desc(su32(sAl) + ks * 256);
                const uint64_t bh = umma_desc(su32(sBh) + ks * 256), bl = umma_desc(su32(sBl) + ks * 256);
                umma_tf32(taddr, ah, bh, idesc, ks > 0);
                umma_tf32(taddr, ah, bl, idesc, 1);
                umma_tf32(taddr, al, bh, idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(mbar)) : "memory");
        }
        ok = __syncthreads_and(mbar_wait(su32(mbar), phase)) != 0;   // one verdict for the whole block
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) {
            if (tid == 0) atomicAdd(&g_wait_timeouts, 1ull);
            break;
        }
        // epilogue: row j of the accumulator is node t0 + j
        const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
        float s = 0.f;
#pragma unroll
        for (int ch = 0; ch < NCH; ch++) {
            if (ch / PER != (warp >> 2)) continue;       // this warp's column group (warp-uniform)
            uint32_t r[16];
            ANOVA_TMEM_LD16(trow + (uint32_t)(16 * ch), r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const int n = 16 * ch + e;
                if (n < R * R) s = fmaf(wx[n / R] * wy[n % R], __uint_as_float(r[e]), s);
            }
        }
        if (kUmmaGroups > 1 && warp >= 4) part[j] = s;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp < 4 && valid) out[W.perm[(int64_t)sp.y + t0 + j]] = kUmmaGroups > 1 ? s + part[j] : s;
    }
    if (!ok) mbar_wait(su32(mbar), phase ^ 1);    // let the tile's MMAs finish before freeing their memory
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        taddr = *tslot;
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kUmmaCols));
    }
}

// shared memory the kernel uses for region size R: A and B heads and tails,
// the partial sums, the mbarrier and the tensor-memory address
constexpr size_t umma_need(int R) {
    return (size_t)(kUmmaTile * 16 * 2 + ((R * R + 15) / 16) * 16 * 16 * 2 + kUmmaTile + kPolyFloats +
                    kUmmaTile * kWPitch) * 4 + 16;
}

template <int R>
static void launch_gather_umma(const int4* sub, int nsub, const DenseWin* descs, int m, const float* poly,
                               cudaStream_t st) {
    constexpr size_t sh = umma_need(R) > kUmmaSmem ? umma_need(R) : kUmmaSmem;   // the floor sets blocks per SM
    static_assert(sh <= 227 * 1024, "shared memory per block");
    static bool attr = [] {
        cudaFuncSetAttribute(k_gather3_umma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        return true;
    }();
    (void)attr;
    k_gather3_umma<R><<<nsub, kUmmaThreads, sh, st>>>(sub, descs, m, poly);
}

anova_status gather3_umma(int R, const int4* sub, int nsub, const DenseWin* descs, int m, const float* poly,
                          cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
    if (kGatherPolyW && (m > 8 || !poly)) {
        set_error("tcgen05 gather: window polynomials missing or m > 8");
        return ANOVA_EINVAL;
    }
    switch (R) {
        case 4: launch_gather_umma<4>(sub, nsub, descs, m, poly, st); break;
        case 6: launch_gather_umma<6>(sub, nsub, descs, m, poly, st); break;
        case 8: launch_gather_umma<8>(sub, nsub, descs, m, poly, st); break;
        case 10: launch_gather_umma<10>(sub, nsub, descs, m, poly, st); break;
        case 12: launch_gather_umma<12>(sub, nsub, descs, m, poly, st); break;
        case 14: launch_gather_umma<14>(sub, nsub, descs, m, poly, st); break;
        case 16: launch_gather_umma<16>(sub, nsub, descs, m, poly, st); break;
        default: set_error("tcgen05 gather: unsupported region size"); return ANOVA_EINVAL;
    }
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// ------------------------------------------------------------- wait probe
// One warp waits on an mbarrier that nothing arrives on, with the bounded poll
// loop of the kernels above cut to `polls` polls, so the wait gives up; the
// block's verdict goes to *gave_up (1 gave up, 0 completed).  No tensor memory,
// no asynchronous copies, no other counter touched.
__global__ void k_wait_probe(int polls, int* gave_up) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1));
    __syncthreads();
    const bool done = __syncthreads_and(mbar_wait(su32(&mbar), 0, polls)) != 0;
    if (threadIdx.x == 0) *gave_up = done ? 0 : 1;
}

unsigned long long* wait_counter() {
    static unsigned long long* addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!addr[dev] && cudaGetSymbolAddress(reinterpret_cast<void**>(&addr[dev]), g_wait_timeouts) != cudaSuccess)
        return nullptr;
    return addr[dev];
}

// The device counter of abandoned waits, read on `st` (stream-ordered, then
// synchronised): a synchronous entry point compares it before and after.
uint64_t wait_timeouts_on(cudaStream_t st) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_wait_timeouts, sizeof(v), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return 0;
    return v;
}

anova_status waits_moved(uint64_t before, cudaStream_t st, const char* who, anova_status s) {
    if (s != ANOVA_OK && s != ANOVA_ENOCONV) return s;
    if (wait_timeouts_on(st) != before) {
        set_error(std::string(who) + ": a bounded wait inside a kernel gave up; the result is invalid");
        return ANOVA_ETIMEOUT;
    }
    return s;
}

}  // namespace anova

extern "C" anova_status anova_debug_wait_probe(int32_t polls, void* stream) {
    if (polls < 1 || polls > anova::kUmmaSpin) {
        anova::set_error("anova_debug_wait_probe: polls must be in 1 .. 2^22");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = nullptr;
    ANOVA_CUDA_TRY(anova::dev_malloc_async((void**)&flag, sizeof(int), st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(flag, 0xff, sizeof(int), st));   // -1: the probe did not run
    anova::k_wait_probe<<<1, 32, 0, st>>>(polls, flag);
    ANOVA_CHECK_LAUNCH();
    int h = -1;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    ANOVA_CUDA_TRY(cudaFreeAsync(flag, st));
    ANOVA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == 1) {
        anova::set_error("anova_debug_wait_probe: the bounded wait gave up");
        return ANOVA_ETIMEOUT;
    }
    if (h == 0) return ANOVA_OK;
    anova::set_error("anova_debug_wait_probe: the probe did not report");
    return ANOVA_ECUDA;
}

extern "C" int64_t anova_wait_timeouts(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, anova::g_wait_timeouts, sizeof(v)) != cudaSuccess) return -1;
    return (int64_t)v;
}
