// dd_tune.cpp -- auto-tuning of the forward kernel's tile shape.
//
// The paper's first experiment (Section IV-A, results Section V-A) runs the
// kernel for every meaningful combination of its four parameters (work-items
// per work-group along time and DM, elements per work-item along time and
// DM) and keeps the configuration with the highest GFLOP/s. Here the sweep
// runs over the compiled variant grid (those four parameters plus the
// staging depth and the channels per stage), skipping variants that do not
// fit the plan or the device. The report carries the statistics of Section
// V-B: mean and standard deviation of GFLOP/s over the variants tried, the
// optimum's distance from the mean in standard deviations ("signal-to-noise
// ratio of the optimum") and Chebyshev's bound 1/k^2 on the chance of
// landing that far from the mean.
#include <chrono>
#include <cmath>
#include <vector>

#include "dd_internal.h"

using namespace dd;

extern "C" dd_status dd_tune(dd_plan p, int32_t budget_ms, dd_tune_report *rep) {
    if (!p) return fail(DD_ERR_ARG, "null plan");
    std::lock_guard<std::mutex> lk(p->mu);
    const size_t in_bytes = size_t(p->B) * p->C * p->stride * elt_bytes(p->dtype);
    const size_t out_bytes = size_t(p->B) * p->D * p->S * 4;
    void *in = nullptr, *w = nullptr, *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&]() {
        if (in) cudaFree(in);
        if (w) cudaFree(w);
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
    };
    cudaError_t e = cudaMalloc(&in, in_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&w, size_t(p->C) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&out, out_bytes);
    if (e == cudaSuccess) e = cudaMemset(in, 0, in_bytes);
    if (e == cudaSuccess) e = cudaMemset(w, 0, size_t(p->C) * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "tuner setup");
    }

    const double flop = double(p->B) * p->D * double(p->S) * p->C;
    const auto wall0 = std::chrono::steady_clock::now();
    std::vector<double> gflops;
    dd_variant best{};
    double best_ms = 1e300;
    const int n = dd_variant_count();
    for (int i = 0; i < n; ++i) {
        if (budget_ms > 0) {
            const double el = std::chrono::duration<double, std::milli>(
                                  std::chrono::steady_clock::now() - wall0)
                                  .count();
            if (el > budget_ms && !gflops.empty()) break;
        }
        dd_variant v;
        dd_variant_get(i, &v);
        FwdTables t;
        if (build_fwd_tables(p, v, &t) != DD_OK) continue;  // does not fit: not meaningful
        dd_status s = launch_forward(p, t, in, w, out, st);  // warm-up
        const int reps = 3;
        if (s == DD_OK) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == DD_OK; ++r) s = launch_forward(p, t, in, w, out, st);
        if (s == DD_OK) e = cudaEventRecord(e1, st);
        if (s == DD_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (s == DD_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        free_fwd_tables(&t);
        if (s != DD_OK || e != cudaSuccess) {
            cleanup();
            return s != DD_OK ? s : cuda_fail(e, "tuner timing");
        }
        const double per = double(ms) / reps;
        gflops.push_back(flop / (per * 1e6));
        if (per < best_ms) {
            best_ms = per;
            best = v;
        }
    }
    cleanup();
    if (gflops.empty()) return fail(DD_ERR_NOT_TUNED, "no variant fits this plan");

    FwdTables t;
    dd_status s = build_fwd_tables(p, best, &t);
    if (s != DD_OK) return s;
    free_fwd_tables(&p->fwd);
    p->fwd = t;

    if (rep) {
        double mean = 0.0, var = 0.0;
        for (double g : gflops) mean += g;
        mean /= double(gflops.size());
        for (double g : gflops) var += (g - mean) * (g - mean);
        const double sd = gflops.size() > 1 ? std::sqrt(var / double(gflops.size() - 1)) : 0.0;
        rep->n_tried = int32_t(gflops.size());
        rep->best = best;
        rep->best_ms = best_ms;
        rep->best_gflops = flop / (best_ms * 1e6);
        rep->mean_gflops = mean;
        rep->std_gflops = sd;
        rep->snr = sd > 0 ? (rep->best_gflops - mean) / sd : 0.0;
        rep->chebyshev = rep->snr > 1.0 ? 1.0 / (rep->snr * rep->snr) : 1.0;
    }
    return DD_OK;
}
