// tc3.cu -- persistent FP32 3-D gather and spread on the fifth-generation
// tensor cores (the NFFT and adjoint NFFT window steps of the fast summation,
// arXiv 2111.10140 Sec. 4.1 Eq. nfft / adjnfft, inside Eq. fastsum of
// Sec. 4.2), for every 3-D window of a plan in one launch.
//
// Work: the plan's merged sub-problem list (bin, first node, count, window),
// split into equal contiguous ranges, one per CTA.  Consecutive sub-problems
// of one bin are one run: their nodes are contiguous in sorted order and they
// share the bin's region (R = Tb + 2m cells per axis starting at bin*Tb - m).
//
// Node weights are evaluated on the fly from the node's cell and offset (no
// per-node weight table): psi(q - m + f), q in [0, 2m), from the plan's
// per-interval FP32 polynomials of the normalised Kaiser-Bessel window, whose
// coefficients travel as a kernel parameter (constant bank, no loads).  Row r
// of the region gets psi(c + m - r + f), c the node's cell inside its bin.
//
// 3xTF32: every operand x is split into head(x) = x truncated to TF32 and
// tail = x - head (exact); head*head + head*tail + tail*head accumulate in
// FP32 in tensor memory (FP32 accuracy: the dropped tail*tail is 2^-20
// relative at most).
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "psi.cuh"
#include "umma.cuh"

namespace anova {

constexpr int kT5Tile = 128;        // nodes per gather tile (MMA M)

// ------------------------------------------------------------------ gather
// Per tile of 128 nodes of a run:
//   U[j][(a,b)] = sum_c wz_j[c] h[a][b][c]     tcgen05.mma M = 128 nodes, N = 16 R
//                                               (row (a, b) at a*16 + b), K = 16
//   s_j = sum_a wx_j[a] sum_b wy_j[b] U[j][(a,b)]   epilogue on the CUDA cores
// Warp roles (13 warps):
//   warps 8-11  producers: thread 256 + j owns node j of a tile.  It copies the
//               node data of the tile three ahead into a ring (cp.async), stages
//               the run's region (B) when a run starts, and writes the tile's
//               operand slot: z weights (A, head and tail), y weights, x data,
//               output index.
//   warp 12     issues the tile's six MMAs (lane 0) into accumulator i mod 2.
//   warps 0-7   consumers: warps w and w + 4 read lanes 32w .. 32w + 31 of the
//               accumulator (node j) and take the first / second half of the
//               region rows a; the halves meet in shared memory.
// Three operand slots, three region buffers, two accumulators.  mbarriers:
//   prod_full[s]  slot s written          (producer, after a named barrier)
//   slot_free[s]  slot s read             (256 consumer threads)
//   acc_full[b]   MMAs of the tile in b done, slot published (commit + issuer)
//   acc_empty[b]  accumulator b read      (256 consumer threads)
// Every wait is bounded; a wait that gives up sets a block-wide abort flag that
// ends the other roles' waits too.
constexpr int kT5Pre = 3;            // tiles of node data copied ahead
constexpr int kT5Ring = kT5Pre + 1;  // ring slots
constexpr int kT5Slots = 3;          // operand slots (and region buffers)
constexpr int kT5YPitch = 20;        // floats per node row of the staged y weights
constexpr int kT5Arr = 7;            // node arrays per tile: fz, cz, fy, cy, fx, cx, perm
constexpr int kT5GThreads = 13 * 32;
constexpr int kT5Rows = 2;
constexpr int kT5SubCache = 512;      // sub-problem entries cached in shared memory           // accumulator rows a per tensor-memory wait in the epilogue

template <int R>
constexpr size_t t5g_smem() {
    return (size_t)(kT5Slots * 2 * R * 16 * 16          // B: [region buffer][head, tail][16 R x 16]
                    + kT5Slots * 2 * kT5Tile * 16       // A: [slot][head, tail][128 x 16]
                    + kT5Slots * kT5Tile * kT5YPitch    // y weights: [slot][128][pitch]
                    + kT5Slots * kT5Tile * 3            // x offset, x cell in the bin, output index: [slot][128]
                    + 2 * kT5Tile                       // partial sums: [tile parity][128]
                    + kT5Ring * kT5Arr * kT5Tile        // node-data ring
                    + 4 * kT5Ring + 4 * kT5SubCache     // ring tiles, sub-problem cache (int4)
                    ) * 4 +
           kT5Slots * 8 * 2 + kT5Slots * 8 * 2 + 2 * 8 * 2 + 32;   // pointers / flags, mbarriers, slot / abort
}

// what a run's window descriptor holds, in registers
struct RunWin {
    const float* frac;
    const int32_t* cell;
    const int32_t* perm;
    const float* grid;
    float* out;
    int64_t N;
    int nos, nb;
};
__device__ __forceinline__ RunWin run_win(const DenseWin* __restrict__ descs, int w) {
    const DenseWin& W = descs[w];
    return RunWin{static_cast<const float*>(W.frac), W.cell, W.perm, static_cast<const float*>(W.grid),
                  static_cast<float*>(W.out), W.N, W.nos, W.nb};
}

template <int R, int M>
__global__ void __launch_bounds__(kT5GThreads, 1)
k_gather3_tc5(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
              const __grid_constant__ PsiCoef<M> P, unsigned long long* __restrict__ timeouts) {
    static_assert(R <= 16 && R > 2 * M, "region up to 16");
    constexpr int NP = R * 16;                           // MMA N: rows (a, b) at a*16 + b
    constexpr int TB = R - 2 * M;
    constexpr int HA = (R + 1) / 2;                      // region rows of the first consumer half
    constexpr uint32_t kCols = 2 * NP <= 256 ? 256u : 512u;
    constexpr uint32_t idesc = umma_idesc_tf32(kT5Tile, NP);
    constexpr int kProd = 256, kIssuer = 384;            // first thread of the producer / issuer warps
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sB = reinterpret_cast<float*>(sm);
    float* sA = sB + kT5Slots * 2 * NP * 16;
    float* sY = sA + kT5Slots * 2 * kT5Tile * 16;
    float* sFx = sY + kT5Slots * kT5Tile * kT5YPitch;
    int* sCx = reinterpret_cast<int*>(sFx + kT5Slots * kT5Tile);
    int* sOut = sCx + kT5Slots * kT5Tile;
    float* part = reinterpret_cast<float*>(sOut + kT5Slots * kT5Tile);
    uint32_t* ring = reinterpret_cast<uint32_t*>(part + 2 * kT5Tile);
    int4* ringTile = reinterpret_cast<int4*>(ring + kT5Ring * kT5Arr * kT5Tile);   // [ring slot] tile
    int4* sCache = ringTile + kT5Ring;                                               // sub-problem cache
    float** sOutp = reinterpret_cast<float**>(sCache + kT5SubCache);
    int64_t* sInfo = reinterpret_cast<int64_t*>(sOutp + kT5Slots);   // per slot: region buffer, or -1 = end
    uint64_t* prod_full = reinterpret_cast<uint64_t*>(sInfo + kT5Slots);
    uint64_t* slot_free = prod_full + kT5Slots;
    uint64_t* acc_full = slot_free + kT5Slots;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

    // tile slots: sub-problem q (at most 256 nodes) is slots 2q and 2q + 1 (nodes 0..127, 128..)
    const int lo = (int)((int64_t)2 * nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)2 * nsub * (blockIdx.x + 1) / gridDim.x);
    if (lo >= hi) return;                                // uniform over the block
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(su32(tslot), kCols);
    if (tid == 0) {
        for (int s = 0; s < kT5Slots; s++) {
            mbar_init(su32(&prod_full[s]), 1);
            mbar_init(su32(&slot_free[s]), 2 * kT5Tile);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(su32(&acc_full[b]), 2);
            mbar_init(su32(&acc_empty[b]), 2 * kT5Tile);
        }
        *abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    auto give_up = [&]() {
        if (atomicExch((int*)abort, 1) == 0 && timeouts) atomicAdd(timeouts, 1ull);
    };

    if (tid >= kProd && tid < kIssuer) {
        // ---------------------------------------------------------------- producers
        // The look-ahead iterator walks the CTA's tile slots kT5Pre tiles ahead: it
        // copies each tile's node data into the ring (cp.async) and writes the tile's
        // (bin, first node, count, window) beside it; sub-problem entries come from a
        // shared-memory cache of the CTA's range.
        const int j = tid - kProd;
        int cache_lo = -1;
        auto sub_at = [&](int q) -> int4 {
            if (cache_lo < 0 || q >= cache_lo + kT5SubCache) {    // uniform: every producer thread walks alike
                bar_sync(1, kT5Tile);
                cache_lo = q;
                const int qe = min((hi + 1) >> 1, q + kT5SubCache);
                for (int k = q + j; k < qe; k += kT5Tile) sCache[k - q] = sub[k];
                bar_sync(1, kT5Tile);
            }
            return sCache[q - cache_lo];
        };
        int pt = lo;                                     // next tile slot of the look-ahead iterator
        int pw = -1;
        RunWin pwin{};
        auto prefetch = [&](int slot) {
            uint32_t* d = ring + slot * kT5Arr * kT5Tile + j;
            int4 tile = make_int4(0, 0, 0, -1);          // w = -1: past the CTA's range
            while (pt < hi) {
                const int4 q = sub_at(pt >> 1);
                const int half = pt & 1;
                pt++;
                const int cnt = q.z - half * kT5Tile;
                if (cnt <= 0) continue;
                const int* live = descs[q.w].live;
                if (live && !*live) continue;
                tile = make_int4(q.x, q.y + half * kT5Tile, min(cnt, kT5Tile), q.w);
                break;
            }
            if (tile.w >= 0) {
                if (tile.w != pw) {
                    pw = tile.w;
                    pwin = run_win(descs, pw);
                }
                const bool v = j < tile.z;
                const int64_t q = v ? (int64_t)tile.y + j : 0;
                const uint32_t nb = v ? 4u : 0u;
                cp_async4(su32(d + 0 * kT5Tile), pwin.frac + 2 * pwin.N + q, nb);
                cp_async4(su32(d + 1 * kT5Tile), pwin.cell + 2 * pwin.N + q, nb);
                cp_async4(su32(d + 2 * kT5Tile), pwin.frac + pwin.N + q, nb);
                cp_async4(su32(d + 3 * kT5Tile), pwin.cell + pwin.N + q, nb);
                cp_async4(su32(d + 4 * kT5Tile), pwin.frac + q, nb);
                cp_async4(su32(d + 5 * kT5Tile), pwin.cell + q, nb);
                cp_async4(su32(d + 6 * kT5Tile), pwin.perm + q, nb);
            }
            if (j == 0) ringTile[slot] = tile;
            cp_async_commit();                           // one group per tile, empty past the end
        };
        for (int t = 0; t < kT5Pre; t++) prefetch(t);
        bar_sync(1, kT5Tile);                            // the first tiles' descriptors are visible
        int cw = -1, cbin = -1;                          // window and bin of the staged region
        RunWin W{};
        int region = -1;
        for (int i = 0;; i++) {
            const int s = i % kT5Slots;
            prefetch((i + kT5Pre) % kT5Ring);           // ends with the named barrier of the last iteration
            if (i >= kT5Slots) {
                const bool w = mbar_wait_abortable(su32(&slot_free[s]), ((i / kT5Slots) - 1) & 1, abort);
                if (!bar_and(1, kT5Tile, w)) {
                    if (j == 0) give_up();
                    break;
                }
            }
            const int4 tile = ringTile[i % kT5Ring];
            if (tile.w < 0) {                            // end marker
                if (j == 0) {
                    sInfo[s] = -1;
                    mbar_arrive(su32(&prod_full[s]), 1);
                }
                break;
            }
            cp_async_wait<kT5Pre>();                     // this thread's copies of tile i have landed
            if (tile.w != cw) W = run_win(descs, tile.w);
            const int bz = tile.x % W.nb, by = (tile.x / W.nb) % W.nb, bx = tile.x / (W.nb * W.nb);
            if (tile.w != cw || tile.x != cbin) {
                // stage the bin's region: row n = a*16 + b of B holds h[a][b][0..R), zero padded
                cw = tile.w;
                cbin = tile.x;
                region++;
                float* bh = sB + (region % kT5Slots) * 2 * NP * 16;
                float* bl = bh + NP * 16;
                const int nos = W.nos;
                const int ox = TB * bx - M, oy = TB * by - M, oz = TB * bz - M;
                for (int u = j; u < NP * 4; u += kT5Tile) {
                    const int n = (u >> 5) * 8 + (u & 7), c0 = 4 * ((u >> 3) & 3);
                    const int a = n >> 4, bb = n & 15;
                    float v[4] = {0.f, 0.f, 0.f, 0.f};
                    if (a < R && bb < R) {
                        const float* row =
                            W.grid + ((size_t)wrap_cell(ox + a, nos) * nos + wrap_cell(oy + bb, nos)) * nos;
#pragma unroll
                        for (int e = 0; e < 4; e++)
                            if (c0 + e < R) v[e] = row[wrap_cell(oz + c0 + e, nos)];
                    }
                    float hh[4], tt[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        hh[e] = tf32_head(v[e]);
                        tt[e] = v[e] - hh[e];
                    }
                    reinterpret_cast<float4*>(bh)[u] = make_float4(hh[0], hh[1], hh[2], hh[3]);
                    reinterpret_cast<float4*>(bl)[u] = make_float4(tt[0], tt[1], tt[2], tt[3]);
                }
            }
            // node j: z weights -> A (head, tail), y weights, x data, output index
            const uint32_t* d = ring + (i % kT5Ring) * kT5Arr * kT5Tile + j;
            const bool valid = j < tile.z;
            float w[16], t[2 * M];
            psi_taps<M>(P, __uint_as_float(d[0 * kT5Tile]), t);
            place_taps<R, M>(t, (int)d[1 * kT5Tile] - TB * bz, w);
            float* ah = sA + s * 2 * kT5Tile * 16;
            float* al = ah + kT5Tile * 16;
#pragma unroll
            for (int kg = 0; kg < 4; kg++) {
                float hh[4], tt[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float x = valid ? w[4 * kg + e] : 0.f;
                    hh[e] = tf32_head(x);
                    tt[e] = x - hh[e];
                }
                const int u = (j >> 3) * 32 + kg * 8 + (j & 7);
                reinterpret_cast<float4*>(ah)[u] = make_float4(hh[0], hh[1], hh[2], hh[3]);
                reinterpret_cast<float4*>(al)[u] = make_float4(tt[0], tt[1], tt[2], tt[3]);
            }
            psi_taps<M>(P, __uint_as_float(d[2 * kT5Tile]), t);
            place_taps<R, M>(t, (int)d[3 * kT5Tile] - TB * by, w);
            float* yrow = sY + (s * kT5Tile + j) * kT5YPitch;
#pragma unroll
            for (int q = 0; q < 4; q++)
                reinterpret_cast<float4*>(yrow)[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            sFx[s * kT5Tile + j] = __uint_as_float(d[4 * kT5Tile]);
            sCx[s * kT5Tile + j] = (int)d[5 * kT5Tile] - TB * bx;
            sOut[s * kT5Tile + j] = valid ? (int)d[6 * kT5Tile] : -1;
            if (j == 0) {
                sOutp[s] = W.out;
                sInfo[s] = region % kT5Slots;
            }
            fence_async_smem();
            bar_sync(1, kT5Tile);
            if (j == 0) mbar_arrive(su32(&prod_full[s]), 1);
        }
        cp_async_wait<0>();
    } else if (tid == kIssuer) {
        // ---------------------------------------------------------------- MMA issuer
        int last_b = -1;
        uint32_t last_parity = 0;
        for (int i = 0;; i++) {
            const int s = i % kT5Slots, b = i & 1;
            if (!mbar_wait_abortable(su32(&prod_full[s]), (i / kT5Slots) & 1, abort)) {
                give_up();
                break;
            }
            const int64_t info = sInfo[s];
            if (i >= 2 && info >= 0 && !mbar_wait_abortable(su32(&acc_empty[b]), ((i >> 1) - 1) & 1, abort)) {
                give_up();
                break;
            }
            if (info < 0) {                              // end marker for the consumers
                if (i >= 2 && !mbar_wait_abortable(su32(&acc_empty[b]), ((i >> 1) - 1) & 1, abort)) {
                    give_up();
                    break;
                }
                mbar_arrive(su32(&acc_full[b]), 2);
                break;
            }
            tc_fence_after();
            const uint32_t a0 = su32(sA + s * 2 * kT5Tile * 16), b0 = su32(sB + (int)info * 2 * NP * 16);
            const uint32_t a1 = a0 + kT5Tile * 16 * 4, b1 = b0 + NP * 16 * 4;
            const uint32_t dd = tbase + (uint32_t)(b * NP);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint64_t dah = umma_desc(a0 + ks * 256), dal = umma_desc(a1 + ks * 256);
                const uint64_t dbh = umma_desc(b0 + ks * 256), dbl = umma_desc(b1 + ks * 256);
                umma_tf32(dd, dah, dbh, idesc, ks > 0);
                umma_tf32(dd, dah, dbl, idesc, 1);
                umma_tf32(dd, dal, dbh, idesc, 1);
            }
            umma_commit(su32(&acc_full[b]));
            mbar_arrive(su32(&acc_full[b]), 1);          // publishes the slot's producer data to the consumers
            last_b = b;
            last_parity = (uint32_t)((i >> 1) & 1);
        }
        // after an abort the MMAs issued last may still run: let them finish (bounded)
        if (last_b >= 0 && *abort) mbar_wait(su32(&acc_full[last_b]), last_parity);
    } else if (tid < kProd) {
        // ---------------------------------------------------------------- consumers
        // One named barrier per tile (all 256 consumers) takes the block's verdict on
        // the accumulator wait and makes the second half's partial sums of the
        // previous tile visible; the first half then writes that tile's results.
        const int h = warp >> 2, j = tid & (kT5Tile - 1);
        const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
        float prev_acc = 0.f;
        int prev_oi = -1;
        float* prev_outp = nullptr;
        for (int i = 0;; i++) {
            const int s = i % kT5Slots, b = i & 1;
            const bool w = mbar_wait_abortable(su32(&acc_full[b]), (i >> 1) & 1, abort);
            const bool ok = bar_and(2, 2 * kT5Tile, w);
            if (h == 0 && prev_oi >= 0) prev_outp[prev_oi] = prev_acc + part[(b ^ 1) * kT5Tile + j];
            if (!ok) {
                if (tid == 0) give_up();
                break;
            }
            tc_fence_after();
            if (sInfo[s] < 0) break;
            float wx[16], wy[16], t[2 * M];
            const float* yrow = sY + (s * kT5Tile + j) * kT5YPitch;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 y4 = reinterpret_cast<const float4*>(yrow)[q];
                wy[4 * q] = y4.x; wy[4 * q + 1] = y4.y; wy[4 * q + 2] = y4.z; wy[4 * q + 3] = y4.w;
            }
            const float fx = sFx[s * kT5Tile + j];
            const int cx = sCx[s * kT5Tile + j];
            const int oi = sOut[s * kT5Tile + j];
            float* outp = sOutp[s];
            mbar_arrive(su32(&slot_free[s]), 1);
            psi_taps<M>(P, fx, t);
            place_taps<R, M>(t, cx, wx);
            const uint32_t tacc = trow + (uint32_t)(b * NP);
            float acc = 0.f;
            auto rows = [&](auto a_lo_c, auto a_hi_c) {
                constexpr int A0 = decltype(a_lo_c)::value, A1 = decltype(a_hi_c)::value;
#pragma unroll
                for (int a0 = A0; a0 < A1; a0 += kT5Rows) {
                    uint32_t u[kT5Rows][16];
#pragma unroll
                    for (int k = 0; k < kT5Rows; k++)
                        if (a0 + k < A1) ANOVA_TMEM_LD16(tacc + (uint32_t)(16 * (a0 + k)), u[k]);
                    tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < kT5Rows; k++) {
                        if (a0 + k >= A1) continue;
                        float e0 = 0.f, e1 = 0.f;
#pragma unroll
                        for (int bb = 0; bb < R; bb += 2) {
                            e0 = fmaf(wy[bb], __uint_as_float(u[k][bb]), e0);
                            if (bb + 1 < R) e1 = fmaf(wy[bb + 1], __uint_as_float(u[k][bb + 1]), e1);
                        }
                        acc = fmaf(wx[a0 + k], e0 + e1, acc);
                    }
                }
            };
            if (h == 0)
                rows(std::integral_constant<int, 0>(), std::integral_constant<int, HA>());
            else
                rows(std::integral_constant<int, HA>(), std::integral_constant<int, R>());
            tc_fence_before();
            mbar_arrive(su32(&acc_empty[b]), 1);
            if (h == 1) {
                part[b * kT5Tile + j] = acc;
            } else {
                prev_acc = acc;
                prev_oi = oi;
                prev_outp = outp;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, kCols);
}

template <int R, int M>
static anova_status launch_gather_tc5(const int4* sub, int nsub, const DenseWin* descs, const float* psi_host,
                                      int sms, cudaStream_t st) {
    constexpr size_t sh = t5g_smem<R>();
    static_assert(sh <= 227 * 1024, "shared memory per block");
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_gather3_tc5<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) ==
               cudaSuccess;
    }();
    if (!attr) {
        set_error("tcgen05 gather: shared-memory attribute refused");
        return ANOVA_ECUDA;
    }
    PsiCoef<M> P;
    std::memcpy(P.c, psi_host, sizeof(P.c));
    const int grid = nsub < sms ? nsub : sms;
    k_gather3_tc5<R, M><<<grid, kT5GThreads, sh, st>>>(sub, nsub, descs, P, wait_counter());
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

// the (R, m) pairs the persistent kernels are built for (Tb = R - 2m even, R <= 16)
bool tc5_supported(int R, int m) {
    return (m == 4 && (R == 10 || R == 12 || R == 14 || R == 16)) || (m == 5 && (R == 12 || R == 14 || R == 16)) ||
           (m == 6 && (R == 14 || R == 16)) || (m == 7 && R == 16);
}

anova_status gather3_tc5(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const float* psi_host,
                         int sms, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
#define ANOVA_G5(R_, M_) \
    if (R == R_ && m == M_) return launch_gather_tc5<R_, M_>(sub, nsub, descs, psi_host, sms, st);
    ANOVA_G5(10, 4) ANOVA_G5(12, 4) ANOVA_G5(14, 4) ANOVA_G5(16, 4)
    ANOVA_G5(12, 5) ANOVA_G5(14, 5) ANOVA_G5(16, 5)
    ANOVA_G5(14, 6) ANOVA_G5(16, 6)
    ANOVA_G5(16, 7)
#undef ANOVA_G5
    set_error("tcgen05 gather: unsupported region size or cutoff");
    return ANOVA_EINVAL;
}

}  // namespace anova

namespace anova {

// ------------------------------------------------------------------ spread
// Per run (consecutive sub-problems of one bin) the region
//   C[(a,b)][c] = sum_p (wx_p[a] wy_p[b]) (alpha_p wz_p[c])
// accumulates in tensor memory over chunks of 32 nodes: tcgen05.mma with
// A = the products wx_p[a] wy_p[b] in tensor memory (row (a, b) at a*16 + b,
// two M tiles of 128 rows; K = the chunk's nodes), B = alpha_p wz_p[c] in
// shared memory (N = 16), D = 2 tiles x 16 columns; 3xTF32 as in the gather.
// Warp roles (13 warps):
//   warps 0-7   A builders: thread (tile w / 4, row 32 (w mod 4) + lane) owns
//               row (a, b); per chunk it forms its row of A from the staged
//               x and y weights and stores heads and tails with tcgen05.st;
//               after a run it reads its row of the accumulator and adds it
//               to the grid (one atomic per region cell and run).
//   warps 8-11  weight warps: warp 8 + k mod 4 takes chunk k (lane = node)
//               and owns weight buffer k mod 4: it forms the node's weights in
//               registers, then (once its buffer is free) writes the x and y
//               weights to shared memory (node-minor rows) and alpha wz
//               (head, tail) as B.
//   warp 12     lane 0 issues the MMAs and closes runs.
// Four weight buffers (one producer each, so every mbarrier phase is waited
// for in order), two A buffers in tensor memory (chunk k mod 2) and two
// accumulators (runs alternate).
constexpr int kS5KC = 32;                      // nodes per chunk (MMA K: 4 steps of 8)
constexpr int kS5Threads = 13 * 32;
constexpr int kS5WWarps = 4;                    // weight warps
constexpr int kS5WPitch = 36;                  // floats per staged weight row (32 nodes + pad)
constexpr uint32_t kS5Cols = 512;              // D: 2 x 32 columns at 0; A: 2 x 128 columns at 64

struct S5Info {                                // one chunk, written by its weight warp
    int w, bin, first, cnt;                    // window, bin, first node, nodes (w < 0: end marker)
};

constexpr size_t s5_smem() {
    return (size_t)(kS5WWarps * 2 * 16 * kS5WPitch     // staged wx, wy rows: [buffer][x, y][16][pitch]
                    + kS5WWarps * 2 * 16 * kS5KC       // B: [buffer][head, tail][16 x 32]
                    ) * 4 +
           kS5WWarps * sizeof(S5Info) + 4 * kT5SubCache * 4 + (2 * kS5WWarps + 4 * 2 + 1) * 8 + 64;
}

template <int R, int M>
__global__ void __launch_bounds__(kS5Threads, 1)
k_spread3_tc5(const int4* __restrict__ sub, int nsub, const DenseWin* __restrict__ descs,
              const __grid_constant__ PsiCoef<M> P, const void* __restrict__ alpha, int alpha_double,
              unsigned long long* __restrict__ timeouts) {
    static_assert(R <= 16 && R > 2 * M, "region up to 16");
    constexpr int TB = R - 2 * M;
    constexpr uint32_t idesc = umma_idesc_tf32(128, 16);
    constexpr uint32_t kSbo = (kS5KC / 4) * 128;          // bytes between 8-row groups of B
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sW = reinterpret_cast<float*>(sm);             // [weight buffer][x, y][16][pitch]
    float* sBm = sW + kS5WWarps * 2 * 16 * kS5WPitch;     // [weight buffer][head, tail][16 x 32]
    S5Info* info = reinterpret_cast<S5Info*>(sBm + kS5WWarps * 2 * 16 * kS5KC);
    int4* sCache = reinterpret_cast<int4*>(info + kS5WWarps);
    uint64_t* wfull = reinterpret_cast<uint64_t*>(sCache + kT5SubCache);   // [4] weight buffer written
    uint64_t* wfree = wfull + kS5WWarps;                  // [4] weights and B of the buffer read
    uint64_t* afull = wfree + kS5WWarps;                  // [2] A of buffer b stored
    uint64_t* afree = afull + 2;                          // [2] A of buffer b read by the MMAs
    uint64_t* dready = afree + 2;                         // [2] accumulator d complete (run closed)
    uint64_t* dfree = dready + 2;                         // [2] accumulator d added to the grid
    uint64_t* drain = dfree + 2;                          // every issued MMA done (after an abort)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

    // chunk slots: sub-problem q is slots 8q .. 8q + 7 (nodes 32 s ..)
    const int lo = (int)((int64_t)8 * nsub * blockIdx.x / gridDim.x);
    const int hi = (int)((int64_t)8 * nsub * (blockIdx.x + 1) / gridDim.x);
    if (lo >= hi) return;                                 // uniform over the block
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(su32(tslot), kS5Cols);
    if (tid == 0) {
        for (int b = 0; b < kS5WWarps; b++) {
            mbar_init(su32(&wfull[b]), 1);
            mbar_init(su32(&wfree[b]), 256 + 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(su32(&afull[b]), 256);
            mbar_init(su32(&afree[b]), 1);
            mbar_init(su32(&dready[b]), 1);
            mbar_init(su32(&dfree[b]), 256);
        }
        mbar_init(su32(drain), 1);
        *abort = 0;
    }
    // every thread walks the chunk sequence alike: sub-problems from a shared cache
    // (filled by all threads before the roles split, reloaded by nobody: the cache
    // holds the CTA's whole range when it fits, else the walk reads global memory)
    const int q_lo = lo >> 3, q_hi = (hi + 7) >> 3;
    const bool cached = q_hi - q_lo <= kT5SubCache;
    if (cached)
        for (int k = q_lo + tid; k < q_hi; k += kS5Threads) sCache[k - q_lo] = sub[k];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    auto give_up = [&]() {
        if (atomicExch((int*)abort, 1) == 0 && timeouts) atomicAdd(timeouts, 1ull);
    };
    auto sub_at = [&](int q) -> int4 { return cached ? sCache[q - q_lo] : sub[q]; };
    // the next non-empty chunk at or after slot *pt; false past the range
    auto next_chunk = [&](int& pt, S5Info& c) -> bool {
        while (pt < hi) {
            const int4 q = sub_at(pt >> 3);
            const int part = pt & 7;
            pt++;
            const int cnt = q.z - part * kS5KC;
            if (cnt <= 0) continue;
            const int* live = descs[q.w].live;
            if (live && !*live) continue;
            c = S5Info{q.w, q.x, q.y + part * kS5KC, min(cnt, kS5KC)};
            return true;
        }
        return false;
    };

    if (warp >= 8 && warp < 8 + kS5WWarps) {
        // ---------------------------------------------------------------- weight warps
        const int me = warp - 8;                          // this warp's chunks: k = me, me + 4, ...
        int pt = lo, k = 0;
        for (;; k++) {
            S5Info c;
            const bool has = next_chunk(pt, c);
            if ((k & (kS5WWarps - 1)) != me) {
                if (!has) break;
                continue;
            }
            const int b = me, use = k >> 2;               // this warp's weight buffer and its use count
            float wx[16], wy[16], wz[16];
            if (has && lane < c.cnt) {
                const DenseWin& W = descs[c.w];
                const int nb = W.nb, bz = c.bin % nb, by = (c.bin / nb) % nb, bx = c.bin / (nb * nb);
                const int64_t pos = (int64_t)c.first + lane, Nn = W.N;
                const float* __restrict__ fr = static_cast<const float*>(W.frac);
                const float fx = fr[pos], fy = fr[Nn + pos], fz = fr[2 * Nn + pos];
                const int cx = W.cell[pos] - TB * bx, cy = W.cell[Nn + pos] - TB * by, cz = W.cell[2 * Nn + pos] - TB * bz;
                float al;
                if (!alpha) al = W.asort[pos];
                else {
                    const int32_t i = W.perm[pos];
                    al = alpha_double ? (float)static_cast<const double*>(alpha)[i] : static_cast<const float*>(alpha)[i];
                }
                float t[2 * M];
                psi_taps<M>(P, fx, t);
                place_taps<R, M>(t, cx, wx);
                psi_taps<M>(P, fy, t);
                place_taps<R, M>(t, cy, wy);
                psi_taps<M>(P, fz, t);
                place_taps<R, M>(t, cz, wz);
#pragma unroll
                for (int r = 0; r < 16; r++) wz[r] *= al;
            } else {
#pragma unroll
                for (int r = 0; r < 16; r++) wx[r] = wy[r] = wz[r] = 0.f;
            }
            // the buffer is free once this warp's previous chunk (k - 4) is consumed
            const bool w = use == 0 || mbar_wait_abortable(su32(&wfree[b]), (use - 1) & 1, abort);
            if (!__all_sync(0xffffffffu, w)) {
                if (lane == 0) give_up();
                break;
            }
            if (!has) {                                   // end marker
                if (lane == 0) {
                    info[b] = S5Info{-1, 0, 0, 0};
                    mbar_arrive(su32(&wfull[b]), 1);
                }
                break;
            }
            float* sx = sW + (b * 2 + 0) * 16 * kS5WPitch;
            float* sy = sW + (b * 2 + 1) * 16 * kS5WPitch;
            float* bh = sBm + (b * 2 + 0) * 16 * kS5KC;
            float* bl = sBm + (b * 2 + 1) * 16 * kS5KC;
#pragma unroll
            for (int r = 0; r < 16; r++) {
                sx[r * kS5WPitch + lane] = wx[r];
                sy[r * kS5WPitch + lane] = wy[r];
                // B: row c = r, column (K) = node lane, K-major core matrices of 8 rows x 4 nodes
                const int o = ((r >> 3) * (kS5KC / 4) + (lane >> 2)) * 32 + (r & 7) * 4 + (lane & 3);
                const float h = tf32_head(wz[r]);
                bh[o] = h;
                bl[o] = wz[r] - h;
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                info[b] = c;
                mbar_arrive(su32(&wfull[b]), 1);
            }
        }
    } else if (warp < 8) {
        // ---------------------------------------------------------------- A builders
        const int t = warp >> 2, row = t * 128 + 32 * (warp & 3) + lane;
        const int a = row >> 4, bb = row & 15;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        int rw = -1, rbin = -1, db = 1, runs = 0;          // the open run and its accumulator
        auto flush = [&](int d, int w, int bin, int use) -> bool {
            // add accumulator d (run `use` of it) to the grid
            if (!__all_sync(0xffffffffu, mbar_wait_abortable(su32(&dready[d]), use & 1, abort))) return false;
            tc_fence_after();
            uint32_t v[16];
            ANOVA_TMEM_LD16(tbase + lane_off + (uint32_t)(d * 32 + t * 16), v);
            tmem_wait_ld();
            tc_fence_before();
            mbar_arrive(su32(&dfree[d]), 1);
            if (a < R && bb < R) {
                const DenseWin& W = descs[w];
                const int nb = W.nb, nos = W.nos, bz = bin % nb, by = (bin / nb) % nb, bx = bin / (nb * nb);
                float* __restrict__ grid = static_cast<float*>(W.grid);
                const size_t rowbase =
                    ((size_t)wrap_cell(TB * bx - M + a, nos) * nos + wrap_cell(TB * by - M + bb, nos)) * nos;
#pragma unroll
                for (int c = 0; c < R; c++) atomicAdd(&grid[rowbase + wrap_cell(TB * bz - M + c, nos)], __uint_as_float(v[c]));
            }
            return true;
        };
        bool ok = true;
        for (int k = 0;; k++) {
            const int b = k & 1, use = k >> 1;            // A buffer and its use count
            const int wb = k & (kS5WWarps - 1);           // weight buffer
            if (!__all_sync(0xffffffffu, mbar_wait_abortable(su32(&wfull[wb]), (k >> 2) & 1, abort))) {
                ok = false;
                break;
            }
            const S5Info c = info[wb];
            if (c.w < 0) {                                // end marker: pass it on to the issuer
                mbar_arrive(su32(&afull[b]), 1);
                break;
            }
            // A of buffer b is free once the MMAs of chunk k - 2 have read it
            if (use >= 1 && !__all_sync(0xffffffffu, mbar_wait_abortable(su32(&afree[b]), (use - 1) & 1, abort))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const float* sx = sW + (wb * 2 + 0) * 16 * kS5WPitch + a * kS5WPitch;
            const float* sy = sW + (wb * 2 + 1) * 16 * kS5WPitch + bb * kS5WPitch;
            const uint32_t acol = tbase + lane_off + (uint32_t)(64 + b * 128 + t * 64);
#pragma unroll
            for (int g = 0; g < kS5KC / 8; g++) {
                uint32_t hv[8], tv[8];
#pragma unroll
                for (int h4 = 0; h4 < 2; h4++) {
                    const float4 x4 = *reinterpret_cast<const float4*>(sx + 8 * g + 4 * h4);
                    const float4 y4 = *reinterpret_cast<const float4*>(sy + 8 * g + 4 * h4);
                    const float2 p0 = __fmul2_rn(make_float2(x4.x, x4.y), make_float2(y4.x, y4.y));
                    const float2 p1 = __fmul2_rn(make_float2(x4.z, x4.w), make_float2(y4.z, y4.w));
                    const float2 h0 = make_float2(tf32_head(p0.x), tf32_head(p0.y));
                    const float2 h1 = make_float2(tf32_head(p1.x), tf32_head(p1.y));
                    const float2 t0 = __fadd2_rn(p0, make_float2(-h0.x, -h0.y));
                    const float2 t1 = __fadd2_rn(p1, make_float2(-h1.x, -h1.y));
                    hv[4 * h4 + 0] = __float_as_uint(h0.x); hv[4 * h4 + 1] = __float_as_uint(h0.y);
                    hv[4 * h4 + 2] = __float_as_uint(h1.x); hv[4 * h4 + 3] = __float_as_uint(h1.y);
                    tv[4 * h4 + 0] = __float_as_uint(t0.x); tv[4 * h4 + 1] = __float_as_uint(t0.y);
                    tv[4 * h4 + 2] = __float_as_uint(t1.x); tv[4 * h4 + 3] = __float_as_uint(t1.y);
                }
                ANOVA_TMEM_ST8(acol + (uint32_t)(8 * g), hv);
                ANOVA_TMEM_ST8(acol + (uint32_t)(32 + 8 * g), tv);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(su32(&wfree[wb]), 1);             // the staged weights of the buffer are read
            mbar_arrive(su32(&afull[b]), 1);
            if (c.w != rw || c.bin != rbin) {
                // chunk k opens a run: the run before it (accumulator db) is closed by the issuer
                if (rw >= 0 && !flush(db, rw, rbin, (runs - 1) >> 1)) {
                    ok = false;
                    break;
                }
                rw = c.w;
                rbin = c.bin;
                db ^= 1;
                runs++;
            }
        }
        if (ok && rw >= 0) ok = flush(db, rw, rbin, (runs - 1) >> 1);
        if (!ok && lane == 0) give_up();
    } else if (warp == 8 + kS5WWarps && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        int rw = -1, rbin = -1, db = 1, runs = 0;
        bool first = true;
        for (int k = 0;; k++) {
            const int b = k & 1, use = k >> 1;
            if (!mbar_wait_abortable(su32(&afull[b]), use & 1, abort)) {
                give_up();
                break;
            }
            const int wb = k & (kS5WWarps - 1);
            const S5Info c = info[wb];
            if (c.w < 0) break;
            if (c.w != rw || c.bin != rbin) {
                if (rw >= 0) umma_commit(su32(&dready[db]));   // close the open run
                rw = c.w;
                rbin = c.bin;
                db ^= 1;
                runs++;
                // accumulator db was last used by run runs - 2: wait until it is in the grid
                if (runs > 2 && !mbar_wait_abortable(su32(&dfree[db]), ((runs - 3) >> 1) & 1, abort)) {
                    give_up();
                    break;
                }
                first = true;
            }
            tc_fence_after();
            const uint32_t b0 = su32(sBm + (wb * 2 + 0) * 16 * kS5KC), b1 = su32(sBm + (wb * 2 + 1) * 16 * kS5KC);
#pragma unroll
            for (int tt = 0; tt < 2; tt++) {
                const uint32_t d = tbase + (uint32_t)(db * 32 + tt * 16);
                const uint32_t ah = tbase + (uint32_t)(64 + b * 128 + tt * 64), al = ah + 32;
#pragma unroll
                for (int ks = 0; ks < kS5KC / 8; ks++) {
                    const uint64_t dbh = umma_desc_sbo(b0 + ks * 256, kSbo), dbl = umma_desc_sbo(b1 + ks * 256, kSbo);
                    umma_tf32_ts(d, ah + 8 * ks, dbh, idesc, (first && ks == 0) ? 0u : 1u);
                    umma_tf32_ts(d, ah + 8 * ks, dbl, idesc, 1);
                    umma_tf32_ts(d, al + 8 * ks, dbh, idesc, 1);
                }
            }
            first = false;
            umma_commit(su32(&afree[b]));
            umma_commit(su32(&wfree[wb]));
        }
        if (!*abort) {
            if (rw >= 0) umma_commit(su32(&dready[db]));   // close the last run
        } else {
            // after an abort the MMAs issued last may still run: let them finish (bounded)
            umma_commit(su32(drain));
            mbar_wait(su32(drain), 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, kS5Cols);
}

template <int R, int M>
static anova_status launch_spread_tc5(const int4* sub, int nsub, const DenseWin* descs, const float* psi_host, int sms,
                                      const void* alpha, int alpha_double, cudaStream_t st) {
    constexpr size_t sh = s5_smem();
    static_assert(sh <= 227 * 1024, "shared memory per block");
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_spread3_tc5<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) ==
               cudaSuccess;
    }();
    if (!attr) {
        set_error("tcgen05 spread: shared-memory attribute refused");
        return ANOVA_ECUDA;
    }
    const int grid = nsub < sms ? nsub : sms;
    k_spread3_tc5<R, M><<<grid, kS5Threads, sh, st>>>(sub, nsub, descs, psi_coef<M>(psi_host), alpha, alpha_double,
                                                      wait_counter());
    ANOVA_CHECK_LAUNCH();
    return ANOVA_OK;
}

anova_status spread3_tc5(int R, int m, const int4* sub, int nsub, const DenseWin* descs, const float* psi_host,
                         int sms, const void* alpha, int alpha_double, cudaStream_t st) {
    if (nsub == 0) return ANOVA_OK;
#define ANOVA_S5(R_, M_) \
    if (R == R_ && m == M_) return launch_spread_tc5<R_, M_>(sub, nsub, descs, psi_host, sms, alpha, alpha_double, st);
    ANOVA_S5(10, 4) ANOVA_S5(12, 4) ANOVA_S5(14, 4) ANOVA_S5(16, 4)
    ANOVA_S5(12, 5) ANOVA_S5(14, 5) ANOVA_S5(16, 5)
    ANOVA_S5(14, 6) ANOVA_S5(16, 6)
    ANOVA_S5(16, 7)
#undef ANOVA_S5
    set_error("tcgen05 spread: unsupported region size or cutoff");
    return ANOVA_EINVAL;
}

}  // namespace anova
