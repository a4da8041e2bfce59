// dd_internal.h -- plan state and kernel-launch interfaces shared by the
// translation units of libdd.so. Not part of the public ABI (see dd.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dd.h"
#include "dd_errbits.h"
#include "dd_kinds.h"

namespace dd {

inline int elt_bytes(dd_dtype t) { return t == DD_F32 ? 4 : (t == DD_U8 ? 1 : 2); }
// Elements per 16 bytes: the TMA bulk-copy granule.
inline int align_elems(dd_dtype t) { return 16 / elt_bytes(t); }

// The streams on which an object's kernels (a plan's, or a batch's) were
// launched, each with an event recorded after its latest launch there.
// Replacing the tables those launches read waits on these events only (the
// host blocks for this object's own work, no device-wide synchronisation).
// Launches made while a stream is being captured into a CUDA graph are not
// tracked; they only mark the object as captured, after which replaced
// tables are kept until the object is destroyed, since a graph may still
// replay launches that read them.
struct LaunchTracker {
    static constexpr int kMax = 8;
    cudaStream_t stream[kMax] = {};
    cudaEvent_t event[kMax] = {};
    unsigned long long used[kMax] = {};  // last note() of each slot
    unsigned long long clock = 0;
    int n = 0;
    bool overflow = false;  // an event call failed: wait() synchronises the device
    bool captured = false;
    std::mutex mu;
    void note(cudaStream_t s);  // call after a successful launch on s
    cudaError_t wait();
    // Orders work queued next on s after every tracked launch (device-side
    // waits on their events; a host wait if an event call failed earlier).
    cudaError_t order_before(cudaStream_t s);
    void destroy();
};

// Input segments of dd_execute_host's copy/compute pipeline.
constexpr int kHostSegments = 8;

// Per-variant staging tables of the forward kernel.
//
// The DM axis is cut into tiles of Dt trials, the time axis into tiles of Ts
// output samples. For DM tile k and channel c, trial d of the tile reads
// input samples [t0 + shift, t0 + shift + Ts) of row c (Section III-B: a 2-D
// work-group shares the union of its trials' inputs). The trials' windows,
// in delay order, are merged while they overlap or touch, and each merged
// window, widened to 16-byte granules, is copied into shared memory once per
// stage (the sub-band kinds always take the whole union [t0 + smin, t0 + smax
// + Ts) as one window). Where neighbouring trials' delays differ by more
// than Ts, a channel thus stages one window per trial rather than a union
// that is mostly gaps.
//
//   copies[k][j][m] = {win_start (elements, relative to t0, 16-byte aligned),
//                      win_len (elements, multiple of 16 bytes; 0 = none),
//                      smem_off (element offset in the stage buffer),
//                      channel - first channel of chunk j}
//                     for the m-th copy of chunk j (capacity n_copies <= 32:
//                     a variant whose chunks need more windows does not fit)
//   offs[k][c][i] = smem element offset of sample t0 of trial k*Dt + i
//                   in channel c (= smem_off + shift - win_start of its window)
struct FwdTables {
    dd_variant v{};
    int Dt = 0, Ts = 0;
    int n_dtiles = 0, n_ttiles = 0;
    int C_pad = 0;               // channels rounded up to chans_per_stage
    int stage_elems = 0;         // data elements in one stage buffer
    int stage_data_bytes = 0;    // rounded to 16
    int stage_offs_bytes = 0;    // chans_per_stage * Dt * 2, rounded to 16
    size_t smem_bytes = 0;       // dynamic shared memory of one CTA
    int4 *d_copies = nullptr;    // [n_dtiles][n_chunks][n_copies]
    int n_copies = 0;
    // launch order of the one-shot kernel: time tiles fastest (true) or DM
    // tiles fastest (false, the default); chosen by dd_tune
    bool time_major = false;
    uint16_t *d_offs = nullptr;
    // sub-band kinds only: d_offs holds per-group trial offsets into the
    // partial-sum buffer, [n_dtiles][C_pad/4][Dt]; d_bdesc the build blocks
    // of every chunk, [n_dtiles][n_chunks][n_blocks] int4 (one block = up to
    // 4 x 32 consecutive elements of one partial series, see
    // build_fwd_tables); p_elems the partial-sum buffer length of one chunk.
    int4 *d_bdesc = nullptr;
    int n_blocks = 0;
    int p_elems = 0;
    // largest delay of each DM tile (over its trials and all channels)
    std::vector<int32_t> dtile_max_shift;
    // stream the device tables were allocated on (stream-ordered; they are
    // freed on it too)
    cudaStream_t aux = nullptr;
    // plans with a declared nonzero input column range only:
    // [n_dtiles][n_ttiles] {first, end} chunks whose staged windows reach it
    // (the hull of those chunks; the others add zeros and are skipped)
    int2 *d_live = nullptr;
};

// Staging choices of the variant grid per (kernel key, CTA shape): 4 chunk
// sizes by 3 pipeline depths, staging depth innermost (dd_variant_get).
constexpr int kStagingChoices = 12;

// Sub-band (kind 2) geometry: channels per group, distinct delay patterns a
// group may have inside one DM tile.
constexpr int kSbGroup = 4;
constexpr int kSbPatterns = 8;

// Adjoint state of a plan, built on first use: the transposed plan (D
// "channels", C "trials", delays max_shift - shift, outputs over the padded
// input rows), the zero-bordered copy of the cotangent it reads, unit
// weights, per (beam, channel) grad_w partial sums, and a G scratch buffer
// for calls that want grad_w without grad_in.
struct AdjState {
    dd_plan_s *plan = nullptr;
    int32_t M = 0;
    float *gpad = nullptr;  // [B][D][plan->stride]
    float *ones = nullptr;  // [D]
    float *part = nullptr;  // [B][C]
    float *gscr = nullptr;  // [B][C][stride], allocated when first needed
};

}  // namespace dd

struct dd_plan_s {
    int32_t C = 0, D = 0, B = 0;
    int64_t S = 0, T_in = 0, stride = 0;
    dd_dtype dtype = DD_F32;
    int32_t max_shift = 0;
    std::vector<int32_t> shifts;  // [D][C]
    // Input columns outside [nz_lo, nz_hi) of every row are known to be zero
    // (set internally for the adjoint's transposed plan, whose input is the
    // zero-bordered cotangent); nz_hi < 0: no such knowledge.
    int64_t nz_lo = 0, nz_hi = -1;

    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;

    dd::FwdTables fwd;
    dd::AdjState adj;
    int32_t *d_shifts = nullptr;  // device copy of `shifts`
    int *d_err = nullptr;         // device error word (dd::kErr* bits)
    // plan-owned stream for table uploads and stream-ordered frees
    cudaStream_t aux = nullptr;
    dd::LaunchTracker launches;
    // tables replaced after a launch of this plan was captured into a graph
    std::vector<dd::FwdTables> retired;

    // device mirrors for dd_execute_host, allocated on first use
    void *h_in_dev = nullptr, *h_w_dev = nullptr, *h_out_dev = nullptr;
    // dd_execute_host's input pipeline: a copy stream, three compute streams
    // and one event per input segment (created on first use)
    cudaStream_t hx_stream[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t hx_event[dd::kHostSegments + 5] = {};

    std::mutex mu;
};

namespace dd {

// Thread-local error reporting (implemented in dd_plan.cpp).
dd_status fail(dd_status s, const std::string &msg);
dd_status cuda_fail(cudaError_t e, const char *what);
dd_status ok();

// Compiled forward variants: (kind, dm_per_thread, samples_per_thread) with a
// kernel for every input type.
struct FwdKernelKey { int kind, dpt, spt; };
const std::vector<FwdKernelKey> &fwd_compiled_keys();
bool fwd_variant_compiled(int kind, int dpt, int spt);

// Builds (or rebuilds) the forward tables for variant v; DD_ERR_ARG if v does
// not fit this plan/device.
dd_status build_fwd_tables(dd_plan_s *p, const dd_variant &v, FwdTables *out);
void free_fwd_tables(FwdTables *t);
// Replaces *cur by next once no tracked launch can still read *cur.
dd_status replace_fwd_tables(dd_plan_s *p, FwdTables *cur, const FwdTables &next);
dd_status check_variant_shape(const dd_variant &v);

// Enqueue the forward kernel with the plan's current tables, over time tiles
// [ttile0, ttile0 + n_ttiles) and DM tiles [dtile0, dtile0 + n_dtiles)
// (-1: to the end).
// CTAs of the plan's forward kernel (variant t) that fit on one SM at once,
// or 0 if the runtime cannot say.
int fwd_resident_per_sm(const dd_plan_s *p, const FwdTables &t);

dd_status launch_forward(dd_plan_s *p, const FwdTables &t, const void *in, const void *w,
                         void *out, cudaStream_t st, int ttile0 = 0, int n_ttiles = -1,
                         int dtile0 = 0, int n_dtiles = -1);

// Adjoint
dd_status ensure_adj_state(dd_plan_s *p);
void free_adj_state(AdjState *a);
dd_status launch_adjoint(dd_plan_s *p, const float *g, const float *w, const float *in,
                         float *gin, float *gw, cudaStream_t st);

bool aligned16(const void *p);

// Tuning cache (DD_TUNE_CACHE): signature of a plan and a record of its
// tuned variant.
std::string plan_signature(const dd_plan_s *p);
void cache_store(const std::string &key, const dd_variant &v, bool time_major);

// Two-pass sweep of the variant grid (dd_tune.cpp). time_ms(v, &ms) sets ms
// <= 0 for variants that do not fit; returns the fastest in *best.
// between_passes (may be empty) sees pass 1's fastest variant before pass 2
// starts (the plan tuner settles the launch order there).
dd_status sweep_variants(int32_t budget_ms, double flop,
                         const std::function<dd_status(const dd_variant &, double *)> &time_ms,
                         dd_variant *best, dd_tune_report *rep,
                         const std::function<dd_status(const dd_variant &)> &between_passes = {});

}  // namespace dd
