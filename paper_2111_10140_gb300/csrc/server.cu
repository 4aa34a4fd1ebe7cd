// server.cu -- a request server for kernel ridge regression with the ANOVA
// fast summation (fit = plan + CG solve of Sec. 2; predict = the test-point
// summation of Sec. 4.3).
//
// Worker threads, each with its own CUDA stream, take requests from one
// queue in arrival order as soon as a worker is idle and the request's device
// memory fits under the budget (continuous admission: a request never waits
// for a batch to fill).  Fits may hold all workers but a quarter (at least
// one), so that predictions -- short by comparison -- never queue behind a
// wall of fits.  Work of different requests overlaps on the GPU.
// Fitted models -- plan and krr_model, whose convolved grids make a
// prediction a binning and a gather -- stay resident on the device until
// released; predictions on one model run concurrently.  Host code only; every computation is a call of the library's
// entry points on the worker's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace anova {

struct ServerRequest {
    int64_t ticket = 0;
    int kind = 0;                 // 0 fit, 1 predict
    // fit
    const double* points = nullptr;
    int64_t N = 0;
    int32_t d = 0;
    std::vector<int32_t> windows;
    int32_t P = 0;
    double ell = 0, eps_B = 0, lambda = 0, tol = 0;
    std::vector<int32_t> n;
    int32_t m = 0, maxit = 0;
    const double* y = nullptr;
    // predict
    int64_t model = 0;
    const double* Z = nullptr;
    int64_t M = 0;
    double* out = nullptr;
    // bookkeeping
    int64_t bytes = 0;
    std::chrono::steady_clock::time_point submitted, started;
    double latency_ms = 0.0;
    anova_status status = ANOVA_OK;
    int32_t iterations = 0;
    double relres = 0.0;
    std::string error;            // the worker's error text, handed to the waiting thread
    bool done = false;
};

struct ServerModel {
    anova_plan* plan = nullptr;
    krr_model* model = nullptr;   // the fitted predictor (its own grids and alpha)
    int64_t N = 0, bytes = 0;
    int32_t d = 0;
    bool ready = false;
    int inflight = 0;             // predictions running on this model
    bool releasing = false;       // released while predictions ran: freed by the last
};

}  // namespace anova

struct anova_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<anova::ServerRequest>> queue;
    std::map<int64_t, std::shared_ptr<anova::ServerRequest>> requests;
    std::map<int64_t, anova::ServerModel> models;
    std::vector<std::thread> workers;
    std::vector<double> latencies;
    int64_t next_ticket = 1;
    int64_t budget = 0, in_use = 0;
    bool stop = false;
    int device = 0;
    int running = 0;
    int running_fits = 0;
    int max_fits = 1;             // workers a fit may occupy; the rest stay free for predictions
    std::chrono::steady_clock::time_point t0;
    // fit admission: nodes of the fits queued and running, and the rate at which
    // the server has been finishing fit nodes (the last completions, all workers together)
    double fit_wait_bound_ms = 0.0;   // 0: no bound
    int64_t fit_nodes_queued = 0, fit_nodes_running = 0;
    double fit_nodes_per_ms = 0.0;    // per worker, over the completed fits (0: none yet)
    int64_t fits_done = 0;
    std::deque<std::pair<std::chrono::steady_clock::time_point, int64_t>> fit_log;   // (completion, N)
    std::deque<std::chrono::steady_clock::time_point> fit_starts;                    // last fit start times
    int fits_queued = 0;
};

namespace anova {

// device bytes of a fitted model: the plan's node arrays, weight tables (FP32
// and the FP64 taps of the mixed plan), grids and work buffers, the CG vectors,
// the coefficients and the model's convolved grids
static int64_t fit_bytes(int64_t N, const std::vector<int32_t>& windows, int32_t P, const std::vector<int32_t>& n,
                         int32_t m) {
    int64_t b = 0;
    for (int l = 0; l < P; l++) {
        int dA = 0;
        while (dA < 3 && windows[3 * l + dA] >= 0) dA++;
        int64_t nos = 2 * (n.empty() ? 32 : n[l]), grid = 1;
        for (int t = 0; t < dA; t++) grid *= nos;
        b += N * (8 * dA + 4 + 4 * dA + 8 * dA + 4 * dA + 64 * dA + 8 + 4 + 8 * dA * (2 * m + 1)) + grid * 8 * 4;
    }
    return b + N * (8 * 5) + (64 << 20);
}

static int64_t predict_bytes(int64_t M, int32_t P) { return M * (P * 8 + 3 * 8 + 48) + (16 << 20); }

static void run_request(anova_server* sv, ServerRequest& r, cudaStream_t st) {
    if (r.kind == 0) {
        ServerModel mdl;
        mdl.N = r.N;
        mdl.d = r.d;
        anova_status s = anova_fastsum_plan(r.points, r.N, r.d, r.d, r.windows.data(), r.P, nullptr, r.ell,
                                            r.n.empty() ? nullptr : r.n.data(), r.m, 2.0, r.eps_B, 8,
                                            ANOVA_MIXED, st, &mdl.plan);
        // no graph capture in server plans: a capture in one worker would make
        // device-wide synchronisation in any other thread of the process fail
        if (s == ANOVA_OK) s = anova_plan_set_graphs(mdl.plan, 0);
        double* alpha = nullptr;
        if (s == ANOVA_OK) {
            if (anova::dev_malloc_async((void**)&alpha, std::max<int64_t>(r.N, 1) * sizeof(double), st) != cudaSuccess)
                s = ANOVA_ENOMEM;
        }
        if (s == ANOVA_OK)
            s = krr_cg_solve(mdl.plan, r.lambda, r.y, alpha, 1, r.N, r.tol, r.maxit, &r.iterations, &r.relres, st);
        if (s == ANOVA_OK || s == ANOVA_ENOCONV) {
            const anova_status sm = krr_model_create(mdl.plan, alpha, st, &mdl.model);
            if (sm != ANOVA_OK) s = sm;
        }
        if (alpha) cudaFreeAsync(alpha, st);
        std::lock_guard<std::mutex> lock(sv->mu);
        if (s == ANOVA_OK || s == ANOVA_ENOCONV) {
            mdl.bytes = r.bytes;
            mdl.ready = true;
            sv->models[r.ticket] = mdl;
        } else {
            krr_model_destroy(mdl.model);
            if (mdl.plan) anova_plan_destroy(mdl.plan);
            sv->in_use -= r.bytes;
        }
        r.status = s;
        if (s != ANOVA_OK) r.error = anova_last_error();
        return;
    }
    ServerModel mdl;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->models.find(r.model);
        if (it == sv->models.end() || !it->second.ready || it->second.inflight == 0) {
            sv->in_use -= r.bytes;
            r.status = ANOVA_EINVAL;
            r.error = "anova_server: the model of this prediction failed to fit or was released";
            return;
        }
        mdl = it->second;
    }
    anova_status s = krr_model_predict(mdl.model, r.Z, r.M, mdl.d, r.out, st);
    if (s != ANOVA_OK) r.error = anova_last_error();
    bool free_now = false;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->in_use -= r.bytes;
        r.status = s;
        auto it = sv->models.find(r.model);
        it->second.inflight--;
        if (it->second.releasing && it->second.inflight == 0) {
            sv->in_use -= it->second.bytes;
            sv->models.erase(it);
            free_now = true;
        }
    }
    if (free_now) {
        krr_model_destroy(mdl.model);
        anova_plan_destroy(mdl.plan);
    }
}

static void worker_main(anova_server* sv) {
    cudaSetDevice(sv->device);
    // predictions on a high-priority stream, fits on a low-priority one: when both
    // have blocks waiting, the GPU schedules the prediction's first, so a
    // prediction's latency does not wait on the fits running beside it
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    cudaStream_t st_pred = nullptr, st_fit = nullptr;
    cudaStreamCreateWithPriority(&st_pred, cudaStreamNonBlocking, prio_high);
    cudaStreamCreateWithPriority(&st_fit, cudaStreamNonBlocking, prio_low);
    cudaStream_t st = st_pred;
    for (;;) {
        std::shared_ptr<ServerRequest> r;
        {
            std::unique_lock<std::mutex> lock(sv->mu);
            for (;;) {
                if (sv->stop) {
                    lock.unlock();
                    cudaStreamDestroy(st_pred);
                    cudaStreamDestroy(st_fit);
                    return;
                }
                // admit the oldest request whose memory fits; a prediction waits
                // while its model is still being fitted
                auto pick = sv->queue.end();
                for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
                    const auto& q = *it;
                    if (q->kind == 1) {
                        auto m = sv->models.find(q->model);
                        if (m == sv->models.end()) {
                            auto rq = sv->requests.find(q->model);
                            const bool fit_over = rq != sv->requests.end() && rq->second->done;
                            if (!fit_over) continue;   // fit still queued or running
                        } else if (!m->second.ready || m->second.releasing) {
                            continue;
                        }
                    } else if (sv->running_fits >= sv->max_fits) {
                        continue;   // predictions behind it may still use the reserved workers
                    }
                    if (sv->in_use + q->bytes <= sv->budget || sv->running == 0) {
                        pick = it;
                        break;
                    }
                    break;   // keep arrival order for memory admission
                }
                if (pick != sv->queue.end()) {
                    r = *pick;
                    sv->queue.erase(pick);
                    sv->in_use += r->bytes;
                    sv->running++;
                    r->started = std::chrono::steady_clock::now();
                    if (r->kind == 0) {
                        sv->running_fits++;
                        sv->fits_queued--;
                        sv->fit_nodes_queued -= r->N;
                        sv->fit_nodes_running += r->N;
                        // a start that had to wait for a worker measures how fast fits drain
                        if (std::chrono::duration<double, std::milli>(r->started - r->submitted).count() > 2.0) {
                            sv->fit_starts.push_back(r->started);
                            if (sv->fit_starts.size() > 16) sv->fit_starts.pop_front();
                        }
                    }
                    if (r->kind == 1) {
                        auto m = sv->models.find(r->model);
                        if (m != sv->models.end()) m->second.inflight++;
                    }
                    break;
                }
                sv->cv_work.wait(lock);
            }
        }
        st = r->kind == 0 ? st_fit : st_pred;
        run_request(sv, *r, st);
        // completion means the result is in device memory
        const cudaError_t se = cudaStreamSynchronize(st);
        if (se != cudaSuccess && r->status == ANOVA_OK) {
            r->status = ANOVA_ECUDA;
            r->error = std::string("anova_server: ") + cudaGetErrorString(se);
        }
        const auto t1 = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            r->latency_ms = std::chrono::duration<double, std::milli>(t1 - r->submitted).count();
            r->done = true;
            sv->running--;
            if (r->kind == 0) {
                sv->running_fits--;
                sv->fit_nodes_running -= r->N;
                const double service = std::chrono::duration<double, std::milli>(t1 - r->started).count();
                if ((r->status == ANOVA_OK || r->status == ANOVA_ENOCONV) && service > 0.0 && r->N > 0) {
                    // running mean of the per-worker fit rate, nodes per millisecond
                    sv->fits_done++;
                    sv->fit_nodes_per_ms += ((double)r->N / service - sv->fit_nodes_per_ms) / (double)sv->fits_done;
                    sv->fit_log.emplace_back(t1, r->N);
                    if (sv->fit_log.size() > 16) sv->fit_log.pop_front();
                }
            }
            if (r->status == ANOVA_OK || r->status == ANOVA_ENOCONV) sv->latencies.push_back(r->latency_ms);
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

static anova_status enqueue(anova_server* sv, std::shared_ptr<ServerRequest> r, int64_t* ticket) {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (r->kind == 0) {
        // Expected wait of this fit before a worker takes it: the fits queued ahead
        // of it (and itself) divided by the rate at which fits that had to wait
        // for a worker have been starting (their last up to 16 starts; the
        // interval up to now counts when none has started for longer than those
        // starts span).  Counting fits rather than nodes makes the estimate follow
        // the mix of fits actually served under the current load.  Until two such
        // starts are recorded the rate is unknown and a fit is taken only if it
        // would not queue.
        if (sv->fit_wait_bound_ms > 0.0) {
            double wait_ms = 0.0;
            const auto now = std::chrono::steady_clock::now();
            const bool would_queue = sv->fits_queued > 0 || sv->running_fits >= sv->max_fits;
            if (would_queue) {
                if (sv->fit_starts.size() >= 2) {
                    const auto first = sv->fit_starts.front(), last = sv->fit_starts.back();
                    const auto end = std::max(last, now - (last - first));
                    const double span = std::chrono::duration<double, std::milli>(end - first).count();
                    const double rate = span > 0.0 ? (double)(sv->fit_starts.size() - 1) / span : 0.0;
                    wait_ms = rate > 0.0 ? (double)(sv->fits_queued + 1) / rate : 1e300;
                } else {
                    wait_ms = 1e300;
                }
            }
            if (wait_ms > sv->fit_wait_bound_ms) {
                set_error("anova_server_submit_fit: expected queue wait " +
                          (wait_ms > 1e18 ? std::string("(unknown: no fit rate measured yet, the fit would queue)")
                                          : std::to_string((int64_t)wait_ms) + " ms") +
                          " exceeds the bound of " + std::to_string((int64_t)sv->fit_wait_bound_ms) + " ms");
                return ANOVA_EBUSY;
            }
        }
        sv->fit_nodes_queued += r->N;
        sv->fits_queued++;
    }
    r->ticket = sv->next_ticket++;
    r->submitted = std::chrono::steady_clock::now();
    sv->requests[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_all();
    return ANOVA_OK;
}

}  // namespace anova

using namespace anova;

extern "C" {

anova_status anova_server_create(int32_t n_workers, int64_t hbm_budget_bytes, anova_server** out) {
    if (!out || n_workers < 1 || n_workers > 64 || hbm_budget_bytes <= 0) {
        set_error("anova_server_create: need 1..64 workers, a positive budget and an output pointer");
        return ANOVA_EINVAL;
    }
    anova_server* sv = new (std::nothrow) anova_server();
    if (!sv) return ANOVA_ENOMEM;
    cudaGetDevice(&sv->device);
    sv->budget = hbm_budget_bytes;
    sv->max_fits = std::max(1, n_workers - std::max(1, n_workers / 4));
    sv->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n_workers; i++) sv->workers.emplace_back(worker_main, sv);
    *out = sv;
    return ANOVA_OK;
}

anova_status anova_server_submit_fit(anova_server* sv, const double* points, int64_t N, int32_t d,
                                     const int32_t* windows, int32_t P, double ell, const int32_t* n, int32_t m,
                                     double eps_B, double lambda, const double* y, double tol, int32_t maxit,
                                     int64_t* ticket) {
    if (!sv || !ticket || !windows || P < 1 || P > kMaxWindows || N < 0 || maxit < 0 ||
        maxit > ANOVA_MAX_CG_ITERS) {
        set_error("anova_server_submit_fit: bad arguments");
        return ANOVA_EINVAL;
    }
    auto r = std::make_shared<ServerRequest>();
    r->kind = 0;
    r->points = points;
    r->N = N;
    r->d = d;
    r->windows.assign(windows, windows + 3 * P);
    r->P = P;
    r->ell = ell;
    if (n) r->n.assign(n, n + P);
    r->m = m;
    r->eps_B = eps_B;
    r->lambda = lambda;
    r->y = y;
    r->tol = tol;
    r->maxit = maxit;
    r->bytes = fit_bytes(N, r->windows, P, r->n, m);
    return enqueue(sv, r, ticket);
}

anova_status anova_server_submit_predict(anova_server* sv, int64_t model, const double* Z, int64_t M, double* out,
                                         int64_t* ticket) {
    if (!sv || !ticket || M < 0) {
        set_error("anova_server_submit_predict: bad arguments");
        return ANOVA_EINVAL;
    }
    int32_t P = 1;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto rq = sv->requests.find(model);
        if (rq == sv->requests.end() || rq->second->kind != 0) {
            set_error("anova_server_submit_predict: unknown model ticket");
            return ANOVA_EINVAL;
        }
        P = rq->second->P;
    }
    auto r = std::make_shared<ServerRequest>();
    r->kind = 1;
    r->model = model;
    r->Z = Z;
    r->M = M;
    r->out = out;
    r->bytes = predict_bytes(M, P);
    return enqueue(sv, r, ticket);
}

anova_status anova_server_wait(anova_server* sv, int64_t ticket, anova_status* result, double* latency_ms,
                               int32_t* iterations, double* relres) {
    if (!sv) return ANOVA_EINVAL;
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) {
        set_error("anova_server_wait: unknown ticket");
        return ANOVA_EINVAL;
    }
    auto r = it->second;
    sv->cv_done.wait(lock, [&] { return r->done; });
    if (result) *result = r->status;
    if (latency_ms) *latency_ms = r->latency_ms;
    if (iterations) *iterations = r->iterations;
    if (relres) *relres = r->relres;
    if (r->status != ANOVA_OK) set_error(r->error);
    if (r->kind == 1) sv->requests.erase(it);   // a fit's record names its model and stays
    return ANOVA_OK;
}

anova_status anova_server_release(anova_server* sv, int64_t model) {
    if (!sv) return ANOVA_EINVAL;
    ServerModel mdl;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->models.find(model);
        if (it == sv->models.end()) {
            set_error("anova_server_release: unknown model");
            return ANOVA_EINVAL;
        }
        if (it->second.inflight > 0) {
            it->second.releasing = true;   // freed by the last running prediction
            return ANOVA_OK;
        }
        mdl = it->second;
        sv->models.erase(it);
        sv->in_use -= mdl.bytes;
    }
    krr_model_destroy(mdl.model);
    anova_plan_destroy(mdl.plan);
    sv->cv_work.notify_all();
    return ANOVA_OK;
}

anova_status anova_server_fit_alpha(anova_server* sv, int64_t fit, double* out, void* stream) {
    if (!sv) return ANOVA_EINVAL;
    krr_model* model = nullptr;
    int64_t N = 0;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->models.find(fit);
        if (it == sv->models.end() || !it->second.ready || it->second.releasing) {
            set_error("anova_server_fit_alpha: unknown, failed or released fit");
            return ANOVA_EINVAL;
        }
        model = it->second.model;
        N = it->second.N;
        it->second.inflight++;             // keeps the model while its coefficients are copied
    }
    anova_status s = (N > 0 && !out) ? ANOVA_EINVAL : krr_model_alpha(model, out, stream);
    if (s == ANOVA_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) s = ANOVA_ECUDA;
    bool free_now = false;
    ServerModel mdl;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->models.find(fit);
        it->second.inflight--;
        if (it->second.releasing && it->second.inflight == 0) {
            mdl = it->second;
            sv->in_use -= mdl.bytes;
            sv->models.erase(it);
            free_now = true;
        }
    }
    if (free_now) {
        krr_model_destroy(mdl.model);
        anova_plan_destroy(mdl.plan);
    }
    if (s == ANOVA_EINVAL) set_error("anova_server_fit_alpha: NULL output");
    return s;
}

anova_status anova_server_set_fit_wait_bound(anova_server* sv, double max_wait_ms) {
    if (!sv || !(max_wait_ms >= 0.0) || !std::isfinite(max_wait_ms)) {
        set_error("anova_server_set_fit_wait_bound: NULL server or a negative or non-finite bound");
        return ANOVA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->fit_wait_bound_ms = max_wait_ms;
    return ANOVA_OK;
}

anova_status anova_server_stats(anova_server* sv, double* p50_ms, double* p99_ms, int64_t* completed,
                                int64_t* bytes_in_use) {
    if (!sv) return ANOVA_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    std::vector<double> v = sv->latencies;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v.empty() ? 0.0 : v[std::min<size_t>(v.size() - 1, (size_t)(f * v.size()))]; };
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
    if (completed) *completed = (int64_t)v.size();
    if (bytes_in_use) *bytes_in_use = sv->in_use;
    return ANOVA_OK;
}

void anova_server_destroy(anova_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        for (auto& q : sv->queue) {
            q->status = ANOVA_EINVAL;
            q->error = "anova_server: the server stopped before this request ran";
            q->done = true;
        }
        sv->queue.clear();
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    for (auto& t : sv->workers) t.join();
    for (auto& kv : sv->models) {
        krr_model_destroy(kv.second.model);
        anova_plan_destroy(kv.second.plan);
    }
    delete sv;
}

}  // extern "C"
