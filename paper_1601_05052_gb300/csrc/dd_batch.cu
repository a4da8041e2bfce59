// dd_batch.cu -- many beams of several observation setups in ONE persistent
// kernel launch, replayed from a CUDA graph.
//
// The paper dedisperses one beam per call and notes that beams are
// independent (Sections II and III-A). Here a batch groups plans of
// different shapes (channels, trial DMs, samples, beams); the work items are
// all (plan, beam, DM tile, time tile) tiles, numbered plan by plan with the
// DM tile fastest. A persistent grid (resident CTAs only) pulls items from a
// device counter with atomicAdd, so uneven setups balance across SMs; plans
// are ordered heaviest tile first so the tail is made of light tiles. One
// launch runs one compiled kernel (kind, DMs and samples per thread) with
// one block size and staging depth, but each plan has its own tile shape
// within it: its split of the trial warps along DM and time (so its DM x
// time tile) and its channels per stage, with its own staging tables; the
// batch tuner picks the common kernel first and then each plan's shape. A
// CTA finishes a tile (every chunk consumed) before it takes the next item,
// so tiles of plans with different slot layouts never overlap in shared
// memory, and the common staging depth keeps the mbarrier phases of
// consecutive tiles in step. The counter reset and the launch form a
// two-node CUDA graph, re-parameterised only when the buffer pointers change.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "dd_fwd_tile.cuh"
#include "dd_internal.h"

namespace dd {

constexpr int kMaxBatchPlans = 16;

struct BatchArgs {
    const FwdArgs *args;  // [n], device
    int n, stages;
    long long item_start[kMaxBatchPlans + 1];
    unsigned long long *counter;
};

template <int KIND, typename T, int DPT, int SPT>
__global__ void __launch_bounds__(fwd_max_threads(KIND), fwd_min_blocks(KIND, DPT, SPT))
    dd_fwd_persistent_kernel(const BatchArgs ba) {
    extern __shared__ __align__(128) unsigned char smem[];
    // The item number alternates between two words: thread 0 writes the
    // next one while a warp that is still leaving the previous tile may not
    // yet have read the current one (a tile with no more chunks than stages
    // lets the staging warp run ahead of the others).
    __shared__ long long s_item[2];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    const volatile int *gave_up = reinterpret_cast<const volatile int *>(&bars[7]);
    fwd_init_barriers<KIND>(bars, ba.stages);
    uint32_t kbase = 0;
    const long long n_items = ba.item_start[ba.n];
    for (int it = 0;; it ^= 1) {
        // a CTA that gave up a wait takes no further items
        if (threadIdx.x == 0)
            s_item[it] = *gave_up ? n_items : (long long)atomicAdd(ba.counter, 1ull);
        __syncthreads();
        const long long item = s_item[it];
        if (item >= n_items) break;
        int i = 0;
        while (item >= ba.item_start[i + 1]) ++i;
        const FwdArgs a = ba.args[i];
        long long loc = item - ba.item_start[i];
        const int dtile = int(loc % a.n_dtiles);
        loc /= a.n_dtiles;
        const int ttile = int(loc % a.n_ttiles);
        const int b = int(loc / a.n_ttiles);
        fwd_tile_any<KIND, T, DPT, SPT>(a, dtile, ttile, b, bars, smem + 128, kbase);
    }
}

namespace {

struct PersistentFn {
    const void *fn = nullptr;
    int (*occupancy)(int block, size_t smem) = nullptr;
};

// Raises the kernel's dynamic shared-memory limit to smem if it is lower (never
// lowers it: another batch's captured graph may launch the same kernel with
// more) and returns its resident CTAs per SM at (block, smem).
template <int KIND, typename T, int DPT, int SPT>
int occupancy_t(int block, size_t smem) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, dd_fwd_persistent_kernel<KIND, T, DPT, SPT>) != cudaSuccess)
        return 0;
    if (size_t(fa.maxDynamicSharedSizeBytes) < smem &&
        cudaFuncSetAttribute(dd_fwd_persistent_kernel<KIND, T, DPT, SPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, dd_fwd_persistent_kernel<KIND, T, DPT, SPT>, block, smem) != cudaSuccess)
        return 0;
    return n;
}

template <typename T>
PersistentFn pick_persistent_t(int kind, int dpt, int spt) {
#define DD_PICK(K_, D_, S_)                                                           \
    if (kind == K_ && dpt == D_ && spt == S_)                                         \
        return PersistentFn{(const void *)&dd_fwd_persistent_kernel<K_, T, D_, S_>, \
                            &occupancy_t<K_, T, D_, S_>};
    DD_FWD_KEYS(DD_PICK)
#undef DD_PICK
    return PersistentFn{};
}

PersistentFn pick_persistent(dd_dtype t, int kind, int dpt, int spt) {
    switch (t) {
        case DD_F32: return pick_persistent_t<float>(kind, dpt, spt);
        case DD_F16: return pick_persistent_t<__half>(kind, dpt, spt);
        case DD_BF16: return pick_persistent_t<__nv_bfloat16>(kind, dpt, spt);
        case DD_U8: return pick_persistent_t<uint8_t>(kind, dpt, spt);
    }
    return PersistentFn{};
}

}  // namespace
}  // namespace dd

struct dd_batch_s {
    std::vector<dd_plan> plans;   // in work-list order (heaviest tile first)
    std::vector<int> user_index;  // position of plans[i] in the caller's arrays
    dd_dtype dtype = DD_F32;
    dd_variant v{};                // the common variant the batch was set to
    std::vector<dd_variant> pv;    // each plan's variant (work-list order)
    std::vector<dd::FwdTables> tabs;
    std::vector<dd::FwdArgs> h_args;
    dd::FwdArgs *d_args = nullptr;
    unsigned long long *d_counter = nullptr;
    dd::BatchArgs ba{};
    size_t smem = 0;
    int grid = 0, block = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool args_on_device = false;
    dd::LaunchTracker launches;
    // tables and graphs replaced after a launch of this batch was captured
    // into a caller's graph (freed with the batch)
    std::vector<dd::FwdTables> retired;
    std::vector<cudaGraphExec_t> retired_exec;
    std::vector<cudaGraph_t> retired_graph;
};

namespace dd {
namespace {

// Drops the batch's tables and graph once none of its launches can still
// read them: waits for the batch's own launches only (no device-wide
// synchronisation); after a capture into a caller's graph they are kept
// until the batch is destroyed.
cudaError_t release_tables(dd_batch_s *bt) {
    const cudaError_t e = bt->launches.wait();
    if (bt->launches.captured) {
        bt->retired.insert(bt->retired.end(), bt->tabs.begin(), bt->tabs.end());
        if (bt->exec) bt->retired_exec.push_back(bt->exec);
        if (bt->graph) bt->retired_graph.push_back(bt->graph);
    } else {
        for (auto &t : bt->tabs) free_fwd_tables(&t);
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
    }
    bt->tabs.clear();
    bt->exec = nullptr;
    bt->graph = nullptr;
    return e;
}

// Per-plan variants can share one persistent launch when they agree on the
// compiled kernel, the staging depth and the number of trial warps.
bool launch_compatible(const dd_variant &a, const dd_variant &b) {
    return a.kind == b.kind && a.dm_per_thread == b.dm_per_thread &&
           a.samples_per_thread == b.samples_per_thread && a.stages == b.stages &&
           a.warps_dm * a.warps_time == b.warps_dm * b.warps_time;
}

// Builds tables, launch shape and graph for the per-plan variants pv (work-
// list order; every plan must fit its variant).
dd_status configure(dd_batch_s *bt, const std::vector<dd_variant> &pv) {
    if (pv.size() != bt->plans.size()) return fail(DD_ERR_ARG, "one variant per plan");
    const dd_variant &v = pv.front();
    for (const dd_variant &x : pv) {
        if (!launch_compatible(v, x))
            return fail(DD_ERR_ARG, "the plans of a batch must share kind, dm_per_thread, "
                                    "samples_per_thread, stages and warps_dm * warps_time");
        dd_status s = check_variant_shape(x);
        if (s != DD_OK) return s;
    }
    PersistentFn pf = pick_persistent(bt->dtype, v.kind, v.dm_per_thread, v.samples_per_thread);
    if (!pf.fn) return fail(DD_ERR_ARG, "variant not compiled");
    std::vector<FwdTables> tabs;
    size_t smem = 0;
    for (size_t i = 0; i < bt->plans.size(); ++i) {
        FwdTables t;
        dd_status s = build_fwd_tables(bt->plans[i], pv[i], &t);
        if (s != DD_OK) {
            for (auto &x : tabs) free_fwd_tables(&x);
            return s;
        }
        smem = std::max(smem, t.smem_bytes);
        tabs.push_back(t);
    }
    const int block = 32 * (v.warps_dm * v.warps_time + extra_warps(v.kind));
    const int occ = pf.occupancy(block, smem);
    if (occ < 1) {
        for (auto &x : tabs) free_fwd_tables(&x);
        return fail(DD_ERR_ARG, "variant does not fit one CTA per SM");
    }
    const cudaError_t we = release_tables(bt);
    bt->tabs = tabs;
    bt->pv = pv;
    bt->smem = smem;
    bt->block = block;
    bt->grid = occ * bt->plans.front()->sm_count;

    const int n = int(bt->plans.size());
    bt->h_args.assign(size_t(n), FwdArgs{});
    bt->ba = BatchArgs{};
    bt->ba.args = bt->d_args;
    bt->ba.n = n;
    bt->ba.stages = v.stages;
    bt->ba.counter = bt->d_counter;
    long long acc = 0;
    for (int i = 0; i < n; ++i) {
        dd_plan p = bt->plans[size_t(i)];
        const FwdTables &t = bt->tabs[size_t(i)];
        FwdArgs &a = bt->h_args[size_t(i)];
        a.C = p->C;
        a.D = p->D;
        a.S = p->S;
        a.stride = p->stride;
        a.Dt = t.Dt;
        a.Ts = t.Ts;
        a.C_pad = t.C_pad;
        a.cch = pv[size_t(i)].chans_per_stage;
        a.stages = pv[size_t(i)].stages;
        a.warps_dm = pv[size_t(i)].warps_dm;
        a.stage_data_bytes = t.stage_data_bytes;
        a.stage_offs_bytes = t.stage_offs_bytes;
        a.n_dtiles = t.n_dtiles;
        a.n_ttiles = t.n_ttiles;
        a.B = p->B;
        a.copies = t.d_copies;
        a.n_copies = t.n_copies;
        a.offs = t.d_offs;
        a.bdesc = t.d_bdesc;
        a.n_blocks = t.n_blocks;
        a.ttile0 = 0;
        a.dtile0 = 0;
        a.grid_tt = t.n_ttiles;
        a.grid_dt = t.n_dtiles;
        a.time_major = 0;  // the persistent kernel orders its own work items
        a.p_elems = t.p_elems;
        a.live = nullptr;  // the persistent kernel sums every chunk
        a.err = p->d_err;
        bt->ba.item_start[i] = acc;
        acc += (long long)t.n_dtiles * t.n_ttiles * p->B;
    }
    bt->ba.item_start[n] = acc;
    bt->args_on_device = false;

    // graph: counter reset -> persistent kernel
    cudaError_t e = cudaGraphCreate(&bt->graph, 0);
    cudaGraphNode_t mset = nullptr, kern = nullptr;
    if (e == cudaSuccess) {
        cudaMemsetParams mp{};
        mp.dst = bt->d_counter;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 2;
        mp.height = 1;
        mp.pitch = 0;
        e = cudaGraphAddMemsetNode(&mset, bt->graph, nullptr, 0, &mp);
    }
    if (e == cudaSuccess) {
        void *params[] = {&bt->ba};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(pf.fn);
        kp.gridDim = dim3(unsigned(bt->grid));
        kp.blockDim = dim3(unsigned(block));
        kp.sharedMemBytes = unsigned(smem);
        kp.kernelParams = params;
        e = cudaGraphAddKernelNode(&kern, bt->graph, &mset, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    if (we != cudaSuccess) return cuda_fail(we, "waiting for the batch's launches");
    return DD_OK;
}

// The same variant for every plan.
dd_status configure(dd_batch_s *bt, const dd_variant &v) {
    dd_status s = configure(bt, std::vector<dd_variant>(bt->plans.size(), v));
    if (s == DD_OK) bt->v = v;
    return s;
}

// Work-list position of the caller's plan index u, or -1.
int worklist_pos(const dd_batch_s *bt, int u) {
    for (size_t i = 0; i < bt->user_index.size(); ++i)
        if (bt->user_index[i] == u) return int(i);
    return -1;
}

double tile_cost(dd_plan p) {
    const FwdTables &t = p->fwd;
    return double(p->C) * t.Dt * t.Ts;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_batch_create(dd_batch *out, int32_t n, const dd_plan *plans) {
    if (!out) return fail(DD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxBatchPlans || !plans)
        return fail(DD_ERR_ARG, "a batch holds 1..16 plans");
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(DD_ERR_ARG, "null plan");
        if (plans[i]->dtype != plans[0]->dtype)
            return fail(DD_ERR_ARG, "the plans of a batch must share the input type");
    }
    auto *bt = new (std::nothrow) dd_batch_s;
    if (!bt) return fail(DD_ERR_NOMEM, "host allocation");
    std::vector<int> idx(static_cast<size_t>(n), 0);
    for (int i = 0; i < n; ++i) idx[size_t(i)] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int x, int y) { return tile_cost(plans[x]) > tile_cost(plans[y]); });
    for (int i : idx) {
        bt->plans.push_back(plans[i]);
        bt->user_index.push_back(i);
    }
    bt->dtype = plans[0]->dtype;
    cudaError_t e = cudaMalloc(&bt->d_args, sizeof(FwdArgs) * size_t(n));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        dd_batch_destroy(bt);
        return cuda_fail(e, "cudaMalloc(batch)");
    }
    // first plan's current variant if every plan fits it, else the defaults
    dd_status s = configure(bt, plans[0]->fwd.v);
    if (s != DD_OK) {
        const int nv = dd_variant_count();
        for (int i = 0; i < nv && s != DD_OK; ++i) {
            dd_variant v;
            dd_variant_get(i, &v);
            if (v.kind == 0 && v.dm_per_thread == 4 && v.samples_per_thread == 4)
                s = configure(bt, v);
        }
        for (int i = 0; i < nv && s != DD_OK; ++i) {
            dd_variant v;
            dd_variant_get(i, &v);
            s = configure(bt, v);
        }
    }
    if (s != DD_OK) {
        dd_batch_destroy(bt);
        return fail(DD_ERR_UNSUPPORTED, "no common variant fits every plan of the batch");
    }
    *out = bt;
    return DD_OK;
}

dd_status dd_batch_execute(dd_batch bt, const void *const *d_in, const void *const *d_w,
                           void *const *d_out, void *stream) {
    if (!bt || !d_in || !d_w || !d_out) return fail(DD_ERR_ARG, "null argument");
    bool changed = !bt->args_on_device;
    for (size_t i = 0; i < bt->plans.size(); ++i) {
        const int u = bt->user_index[i];
        if (!d_in[u] || !d_w[u] || !d_out[u]) return fail(DD_ERR_ARG, "null buffer");
        if (!aligned16(d_in[u]) || !aligned16(d_w[u]) || !aligned16(d_out[u]))
            return fail(DD_ERR_ARG, "device pointers must be 16-byte aligned");
        FwdArgs &a = bt->h_args[i];
        if (a.in != d_in[u] || a.w != d_w[u] || a.out != d_out[u]) changed = true;
        a.in = d_in[u];
        a.w = d_w[u];
        a.out = d_out[u];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (changed) {
        // the batch's earlier launches (on any stream) read the old arguments
        e = bt->launches.order_before(st);
        if (e != cudaSuccess) return cuda_fail(e, "ordering after the batch's launches");
        e = cudaMemcpyAsync(bt->d_args, bt->h_args.data(), sizeof(FwdArgs) * bt->h_args.size(),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch args upload");
        bt->args_on_device = true;
    }
    e = cudaGraphLaunch(bt->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batch)");
    bt->launches.note(st);
    return DD_OK;
}

dd_status dd_batch_get_variant(dd_batch bt, dd_variant *v) {
    if (!bt || !v) return fail(DD_ERR_ARG, "null argument");
    *v = bt->v;
    return DD_OK;
}

dd_status dd_batch_set_variant(dd_batch bt, const dd_variant *v) {
    if (!bt || !v) return fail(DD_ERR_ARG, "null argument");
    dd_status s = check_variant_shape(*v);
    if (s != DD_OK) return s;
    return configure(bt, *v);  // waits for the batch's own launches before replacing
}

dd_status dd_batch_get_plan_variant(dd_batch bt, int32_t i, dd_variant *v) {
    if (!bt || !v) return fail(DD_ERR_ARG, "null argument");
    const int j = worklist_pos(bt, i);
    if (j < 0) return fail(DD_ERR_ARG, "plan index out of range");
    *v = bt->pv[size_t(j)];
    return DD_OK;
}

dd_status dd_batch_set_plan_variant(dd_batch bt, int32_t i, const dd_variant *v) {
    if (!bt || !v) return fail(DD_ERR_ARG, "null argument");
    const int j = worklist_pos(bt, i);
    if (j < 0) return fail(DD_ERR_ARG, "plan index out of range");
    std::vector<dd_variant> pv = bt->pv;
    pv[size_t(j)] = *v;
    for (const dd_variant &x : pv)
        if (!launch_compatible(x, *v))
            return fail(DD_ERR_ARG, "the plans of a batch must share kind, dm_per_thread, "
                                    "samples_per_thread, stages and warps_dm * warps_time");
    const std::vector<dd_variant> old = bt->pv;
    dd_status s = configure(bt, pv);
    if (s != DD_OK) {
        const dd_status keep = dd_get_last_error();
        const std::string msg = dd_last_error_message();
        configure(bt, old);  // the previous variants fitted; keep them
        return fail(keep, msg);
    }
    return DD_OK;
}

dd_status dd_batch_tune(dd_batch bt, int32_t budget_ms, dd_tune_report *rep) {
    if (!bt) return fail(DD_ERR_ARG, "null batch");
    const size_t n = bt->plans.size();
    std::vector<void *> ins(n, nullptr), ws(n, nullptr), outs(n, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    double flop = 0.0;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        dd_plan p = bt->plans[i];
        const size_t ib = size_t(p->B) * p->C * p->stride * elt_bytes(p->dtype);
        e = cudaMalloc(&ins[i], ib);
        if (e == cudaSuccess) e = cudaMemset(ins[i], 0, ib);
        if (e == cudaSuccess) e = cudaMalloc(&ws[i], size_t(p->C) * 4);
        if (e == cudaSuccess) e = cudaMemset(ws[i], 0, size_t(p->C) * 4);
        if (e == cudaSuccess) e = cudaMalloc(&outs[i], size_t(p->B) * p->D * p->S * 4);
        flop += double(p->B) * p->D * double(p->S) * p->C;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    auto cleanup = [&]() {
        for (size_t i = 0; i < n; ++i) {
            if (ins[i]) cudaFree(ins[i]);
            if (ws[i]) cudaFree(ws[i]);
            if (outs[i]) cudaFree(outs[i]);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        bt->args_on_device = false;
    };
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "batch tuner setup");
    }
    // arrays in the caller's order
    std::vector<const void *> uin(n), uw(n);
    std::vector<void *> uout(n);
    for (size_t i = 0; i < n; ++i) {
        const int u = bt->user_index[i];
        uin[size_t(u)] = ins[i];
        uw[size_t(u)] = ws[i];
        uout[size_t(u)] = outs[i];
    }
    auto time_pv = [&](const std::vector<dd_variant> &pv, double *ms) -> dd_status {
        if (configure(bt, pv) != DD_OK) return DD_OK;  // does not fit every plan
        bt->args_on_device = false;
        dd_status s = dd_batch_execute(bt, uin.data(), uw.data(), uout.data(), st);
        const int reps = 3;
        cudaError_t ce = cudaSuccess;
        if (s == DD_OK) ce = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == DD_OK && ce == cudaSuccess; ++r)
            s = dd_batch_execute(bt, uin.data(), uw.data(), uout.data(), st);
        if (s == DD_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (s == DD_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float f = 0.f;
        if (s == DD_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&f, e0, e1);
        if (s != DD_OK) return s;
        if (ce != cudaSuccess) return cuda_fail(ce, "batch tuner timing");
        *ms = double(f) / reps;
        return DD_OK;
    };
    auto time_ms = [&](const dd_variant &v, double *ms) -> dd_status {
        return time_pv(std::vector<dd_variant>(n, v), ms);
    };
    const auto wall0 = std::chrono::steady_clock::now();
    const dd_variant start = bt->v;
    dd_variant best = start;
    dd_status s = sweep_variants(budget_ms, flop, time_ms, &best, rep);
    // Per-setup tile shapes: with the common kernel and staging depth fixed,
    // each plan in turn tries every split of the trial warps along DM and
    // time and every chunk size, keeping what shortens the whole launch by
    // more than 1 % (the paper's finding that no one configuration suits
    // every setup, applied within one launch).
    std::vector<dd_variant> pv(n, best);
    if (s == DD_OK && n > 1) {
        double cur = -1.0;
        s = time_pv(pv, &cur);
        const int tw = best.warps_dm * best.warps_time;
        auto over = [&]() {
            return budget_ms > 0 && std::chrono::duration<double, std::milli>(
                                        std::chrono::steady_clock::now() - wall0)
                                            .count() > 2.0 * budget_ms;
        };
        for (size_t j = 0; j < n && s == DD_OK && cur > 0 && !over(); ++j) {
            for (int wdm = 1; wdm <= tw && s == DD_OK; ++wdm) {
                if (tw % wdm) continue;
                for (int cch : {4, 8, 16, 32}) {
                    std::vector<dd_variant> cand = pv;
                    cand[j].warps_dm = wdm;
                    cand[j].warps_time = tw / wdm;
                    cand[j].chans_per_stage = cch;
                    if (cand[j].warps_dm == pv[j].warps_dm && cand[j].chans_per_stage == cch)
                        continue;
                    double ms = -1.0;
                    s = time_pv(cand, &ms);
                    if (s != DD_OK) break;
                    if (ms > 0 && ms < 0.99 * cur) {
                        cur = ms;
                        pv = cand;
                    }
                }
            }
        }
    }
    cleanup();
    dd_status s2 = s == DD_OK ? configure(bt, pv) : configure(bt, start);
    if (s2 == DD_OK) bt->v = s == DD_OK ? best : start;
    if (s != DD_OK) return s;
    return s2;
}

void dd_batch_destroy(dd_batch bt) {
    if (!bt) return;
    bt->launches.captured = false;  // the batch and every graph of its launches end here
    release_tables(bt);
    for (auto &t : bt->retired) free_fwd_tables(&t);
    for (cudaGraphExec_t x : bt->retired_exec) cudaGraphExecDestroy(x);
    for (cudaGraph_t g : bt->retired_graph) cudaGraphDestroy(g);
    bt->launches.destroy();
    if (bt->d_args) cudaFree(bt->d_args);
    if (bt->d_counter) cudaFree(bt->d_counter);
    delete bt;
}

}  // extern "C"
