// autotune.cu -- choice of the bin side per window dimension by measurement.
//
// The dense spread / gather kernels cut every window's grid into bins of
// Tb^dA cells; a sub-problem is one bin's nodes and its region of (Tb + 2m)^dA
// cells.  Larger bins mean fewer, larger regions (fewer grid atomics per node,
// more weight-table work per region), smaller bins the opposite; which is
// faster depends on N, n and m.  anova_autotune_bins builds the plan with the
// default rule, then tries each admissible bin side for the 1-D, the 2-D and
// the 3-D windows in turn (coordinate descent, the other dimensions held at
// their best so far), timing the matrix-vector product with CUDA events, and
// returns the fastest choice.  anova_autotune_kernels then picks, on a built
// plan, the form of the 3-D spread and gather kernels and the schedule of the
// 1-D / 2-D windows against the 3-D ones, also by timing.  The paper fixes no
// binning or kernel form; these are tuning steps of the GPU design only.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace anova {

template <typename T>
__global__ void k_tune_fill(T* a, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (T)(((i * 2654435761ull) >> 7) % 2001) * (T)1e-3 - (T)1;
}

}  // namespace anova

using namespace anova;

extern "C" anova_status anova_autotune_bins(const double* points, int64_t N, int32_t d, int64_t ld,
                                            const int32_t* windows, int32_t P, const double* weights, double ell,
                                            const int32_t* n, int32_t m, double sigma, double eps_B, int32_t p,
                                            int32_t precision, int32_t reps, int32_t* bin_side, double* ms,
                                            void* stream) {
    if (!bin_side || reps < 1 || N < 1 || !windows || P < 1) {
        set_error("anova_autotune_bins: need N >= 1, windows, reps >= 1 and an output array");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = (precision & ANOVA_FP32) != 0;
    const int32_t dtype = f32 ? ANOVA_FP32 : ANOVA_FP64;
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    bool present[3] = {false, false, false};
    for (int l = 0; l < P; l++) {
        int dA = 0;
        while (dA < 3 && windows[3 * l + dA] >= 0) dA++;
        if (dA >= 1) present[dA - 1] = true;
    }
    void *alpha = nullptr, *out = nullptr;
    Scratch scratch(st, false);
    ANOVA_CUDA_TRY(scratch.alloc(&alpha, N * esz));
    ANOVA_CUDA_TRY(scratch.alloc(&out, N * esz));
    if (f32) k_tune_fill<float><<<grid_for(N, kThreads, 1024), kThreads, 0, st>>>((float*)alpha, N);
    else k_tune_fill<double><<<grid_for(N, kThreads, 1024), kThreads, 0, st>>>((double*)alpha, N);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // time one configuration; false if the plan does not take the requested sides
    auto timed = [&](const int32_t* sides, double* t_ms) -> anova_status {
        anova_plan* plan = nullptr;
        ANOVA_TRY(anova_fastsum_plan_bins(points, N, d, ld, windows, P, weights, ell, n, m, sigma, eps_B, p,
                                          precision, sides, stream, &plan));
        bool honoured = true;
        for (int l = 0; l < P && sides; l++) {
            const WindowPlan& w = plan->win[l];
            if (sides[w.dA - 1] > 0 && (!w.dense || w.T != sides[w.dA - 1])) honoured = false;
        }
        anova_status s = ANOVA_OK;
        if (honoured) {
            for (int k = 0; k < 3 && s == ANOVA_OK; k++) s = anova_matvec(plan, dtype, alpha, out, 1, N, stream);
            if (s == ANOVA_OK) {
                cudaEventRecord(e0, st);
                for (int k = 0; k < reps && s == ANOVA_OK; k++) s = anova_matvec(plan, dtype, alpha, out, 1, N, stream);
                cudaEventRecord(e1, st);
                float t = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                    s = ANOVA_ECUDA;
                *t_ms = (double)t / reps;
            }
        } else {
            *t_ms = -1.0;
        }
        anova_plan_destroy(plan);
        return s;
    };
    int32_t best[3] = {0, 0, 0};
    double best_ms = 0.0;
    anova_status s = timed(best, &best_ms);
    for (int dim = 1; dim <= 3 && s == ANOVA_OK; dim++) {
        if (!present[dim - 1]) continue;
        for (int Tb = 2; Tb + 2 * m <= 16 && s == ANOVA_OK; Tb += 2) {
            int32_t trial[3] = {best[0], best[1], best[2]};
            trial[dim - 1] = Tb;
            double t = 0.0;
            s = timed(trial, &t);
            if (s == ANOVA_OK && t > 0.0 && t < best_ms) {
                best_ms = t;
                for (int k = 0; k < 3; k++) best[k] = trial[k];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ANOVA_OK) return s;
    for (int k = 0; k < 3; k++) bin_side[k] = best[k];
    if (ms) *ms = best_ms;
    return ANOVA_OK;
}

namespace {

// the plan's current kernel forms: 3-D spread, 3-D gather, 1-D / 2-D schedule
void current_forms(const anova_plan* plan, int32_t c[3]) {
    c[0] = plan->spread_tc ? (plan->spread_f16 ? 3 : (plan->spread_pipe ? 2 : 1)) : 0;
    c[1] = plan->gather_tc ? (plan->gather_umma ? (plan->gather_tc5 ? 3 : 2) : 1) : 0;
    c[2] = plan->overlap12 & 3;
}

void apply_forms(anova_plan* plan, const int32_t c[3]) {
    plan->spread_tc = c[0] >= 1;
    plan->spread_pipe = c[0] >= 2;
    plan->spread_f16 = c[0] == 3;
    plan->spread_tc5 = false;
    plan->gather_tc = c[1] >= 1;
    plan->gather_umma = c[1] >= 2;
    plan->gather_tc5 = c[1] >= 3;
    plan->overlap12 = c[2] == 0 ? 0 : (plan->overlap12 & 4) | c[2];   // the stream priority bit is kept
    for (auto& g : plan->graphs)       // the captured launch sequences hold the old kernels
        if (g.exec) cudaGraphExecDestroy(g.exec);
    plan->graphs.clear();
}

}  // namespace

extern "C" anova_status anova_plan_set_kernels(anova_plan* plan, const int32_t* forms) {
    if (!plan || !forms || forms[0] < 0 || forms[0] > 3 || forms[1] < 0 || forms[1] > 3 || forms[2] < 0 ||
        forms[2] > 3) {
        set_error("anova_plan_set_kernels: forms must be spread 0..3, gather 0..3, schedule 0..3");
        return ANOVA_EINVAL;
    }
    apply_forms(plan, forms);
    return ANOVA_OK;
}

extern "C" anova_status anova_plan_get_kernels(const anova_plan* plan, int32_t* forms) {
    if (!plan || !forms) {
        set_error("anova_plan_get_kernels: NULL argument");
        return ANOVA_EINVAL;
    }
    current_forms(plan, forms);
    return ANOVA_OK;
}

extern "C" anova_status anova_autotune_kernels(anova_plan* plan, int32_t reps, int32_t* choice, double* ms,
                                               void* stream) {
    if (!plan || !choice || reps < 1) {
        set_error("anova_autotune_kernels: need a plan, reps >= 1 and an output array");
        return ANOVA_EINVAL;
    }
    if (!(plan->precision & ANOVA_FP32) || plan->N < 1) {
        set_error("anova_autotune_kernels: the plan must hold the FP32 operator and at least one node");
        return ANOVA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = plan->N;
    float *alpha = nullptr, *out = nullptr;
    Scratch scratch(st, false);
    ANOVA_CUDA_TRY(scratch.alloc(&alpha, N * sizeof(float)));
    ANOVA_CUDA_TRY(scratch.alloc(&out, N * sizeof(float)));
    k_tune_fill<float><<<grid_for(N, kThreads, 1024), kThreads, 0, st>>>(alpha, N);
    ANOVA_CHECK_LAUNCH();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ANOVA_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("anova_autotune_kernels: cudaEventCreate failed");
        return ANOVA_ECUDA;
    }
    int32_t start[3];
    current_forms(plan, start);
    auto timed = [&](const int32_t* c, double* t_ms) -> anova_status {
        apply_forms(plan, c);
        for (int k = 0; k < 2; k++) ANOVA_TRY(anova_matvec(plan, ANOVA_FP32, alpha, out, 1, N, stream));
        ANOVA_CUDA_TRY(cudaEventRecord(e0, st));
        for (int k = 0; k < reps; k++) ANOVA_TRY(anova_matvec(plan, ANOVA_FP32, alpha, out, 1, N, stream));
        ANOVA_CUDA_TRY(cudaEventRecord(e1, st));
        float t = 0.f;
        ANOVA_CUDA_TRY(cudaEventSynchronize(e1));
        ANOVA_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        *t_ms = (double)t / reps;
        return ANOVA_OK;
    };
    // coordinate descent from the plan's current forms
    int32_t best[3] = {start[0], start[1], start[2]};
    double best_ms = 0.0;
    anova_status s = timed(best, &best_ms);
    const int nform[3] = {4, 4, 4};
    for (int k = 0; k < 3 && s == ANOVA_OK; k++)
        for (int v = 0; v < nform[k] && s == ANOVA_OK; v++) {
            if (v == best[k]) continue;
            int32_t trial[3] = {best[0], best[1], best[2]};
            trial[k] = v;
            double t = 0.0;
            s = timed(trial, &t);
            if (s == ANOVA_OK && t < best_ms) {
                best_ms = t;
                best[k] = v;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_forms(plan, s == ANOVA_OK ? best : start);
    if (s != ANOVA_OK) return s;
    for (int k = 0; k < 3; k++) choice[k] = best[k];
    if (ms) *ms = best_ms;
    return ANOVA_OK;
}
