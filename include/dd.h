/*
 * dd.h -- C ABI of the GB300 (sm_103a) brute-force dedispersion library
 * (libdd.so).
 *
 * The operation (Algorithm 1 of Sclocco et al., "Auto-Tuning Dedispersion for
 * Many-Core Accelerators", Section III-A, with per-channel weights):
 *
 *     out[b][d][t] = sum_{c=0}^{C-1} w[c] * in[b][c][t + shift[d][c]]
 *
 * for beam b < B, trial DM d < D, output sample t < S. The delay table comes
 * from Eq. 1 (Section II): shift[d][c] = round(K * DM_d * (f_c^-2 - f_ref^-2)
 * / t_samp) with K = 4.148808e3 MHz^2 pc^-1 cm^3 s, frequencies in MHz,
 * t_samp in seconds, rounded to nearest with halves away from zero, evaluated
 * in FP64 on the host as ((K * DM) * (1/(f*f) - 1/(f_ref*f_ref))) / t_samp.
 *
 * Conventions shared by every entry point:
 *   - Layout. Input rows are [B][C][stride] elements of the plan's input type,
 *     where stride = dd_plan_input_stride(plan) >= T_in = S + max shift and
 *     stride * sizeof(element) is a multiple of 16 bytes. Only the first T_in
 *     entries of a row are read as data (the kernel may load pad entries into
 *     shared memory but never sums them). Output is [B][D][S], contiguous.
 *   - Types. DD_F32, DD_F16, DD_BF16 inputs take float weights and produce
 *     float32 output (FP32 accumulation). DD_U8 input takes int32 weights and
 *     produces int32 output, exact integer arithmetic; the caller keeps
 *     |w| * 255 * C below 2^31.
 *   - Ownership. The caller owns every input/output buffer and stream. A plan
 *     owns its host and device tables only. Device pointers must be 16-byte
 *     aligned, else DD_ERR_ARG.
 *   - Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream). Device work is asynchronous: errors raised by a kernel
 *     surface at a later call or through dd_plan_check_device().
 *   - Errors. Every call returns a dd_status; the last failure's message is
 *     kept per thread (dd_last_error_message). No call throws or aborts.
 *   - Threads. A plan may be used from several threads and streams at once
 *     for dd_execute. dd_adjoint and dd_execute_host use plan-owned device
 *     buffers, so their calls on one plan must be ordered (one stream, one
 *     thread at a time); dd_tune, dd_tune_adjoint, the set_variant calls and
 *     dd_plan_set_launch_order must not run concurrently with other calls on
 *     the same plan.
 */
#ifndef DD_H_
#define DD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DD_VERSION 1

typedef enum { DD_F32 = 0, DD_F16 = 1, DD_BF16 = 2, DD_U8 = 3 } dd_dtype;

typedef enum {
    DD_OK = 0,
    DD_ERR_ARG = 1,          /* invalid argument (null, size, alignment, order) */
    DD_ERR_CUDA = 2,         /* a CUDA runtime call failed (no device, launch error) */
    DD_ERR_NOMEM = 3,        /* device or host allocation failed */
    DD_ERR_UNSUPPORTED = 4,  /* valid request this build does not implement */
    DD_ERR_TIMEOUT = 5,      /* a kernel gave up a bounded wait (device error word) */
    DD_ERR_NOT_TUNED = 6,    /* no tuned variant recorded for this plan */
    DD_ERR_DEVICE = 7        /* a kernel reported another device-side error */
} dd_status;

typedef struct dd_plan_s *dd_plan;
typedef struct dd_batch_s *dd_batch;
typedef struct dd_stream_s *dd_stream;

/* Tile shape of the forward kernel (Section III-B's four parameters plus the
 * staging pipeline). A CTA computes dm_per_thread * warps_dm trial DMs by
 * 32 * samples_per_thread * warps_time output samples; input rows of
 * chans_per_stage channels are staged per pipeline stage, `stages` deep.
 * kind 0: lane l of a warp owns samples l, l+32, ...; each add reads its
 *         input from shared memory.
 * kind 1: a thread owns samples_per_thread (odd) consecutive samples and
 *         keeps, per channel, the union window of its warp's trials in
 *         registers, serving every trial of the warp from it.
 * kind 2: sub-band partial sums: per group of 4 adjacent channels the CTA
 *         builds, once per chunk, the weighted 4-channel sum series of each
 *         distinct relative delay pattern of its trials, and every trial adds
 *         one series value per group (lane-strided); plus one producer warp.
 * kind 3: kind 2 with 4 dedicated builder warps (warp-specialised).
 * kind 4: kind 2 in CTAs of up to 16 trial warps (one CTA per SM).
 * kind 5: kind 0 that reuses the loaded operands for a trial whose delay in
 *         the channel equals the previous trial's.
 * kind 6: kind 4 with one partial-sum slot and a second barrier per chunk,
 *         so that FP32 input fits chunks of 32 channels.
 * Results do not depend on the variant beyond FP32 summation order (8-bit
 * input: bit-identical). */
typedef struct {
    int32_t kind;                /* 0..6, see above                         */
    int32_t dm_per_thread;       /* DMs accumulated per thread (registers) */
    int32_t samples_per_thread;  /* samples accumulated per thread          */
    int32_t warps_dm;            /* warps along the DM axis of a CTA        */
    int32_t warps_time;          /* warps along the time axis of a CTA      */
    int32_t chans_per_stage;     /* channels per pipeline stage: 4, 8, 16, 32 */
    int32_t stages;              /* shared-memory pipeline depth (2..4)     */
} dd_variant;

/* Outcome of an auto-tuning sweep (Section IV-A / V-B of the paper). Times
 * are mean CUDA-event milliseconds per launch; `gflops` counts one add per
 * channel per output (B*D*S*C flop). snr = (best - mean) / std of the GFLOP/s
 * over the variants tried; chebyshev = 1/snr^2, the bound on the chance that a
 * configuration picked at random performs that far above the mean. */
typedef struct {
    int32_t n_tried;
    dd_variant best;
    double best_ms;
    double best_gflops;
    double mean_gflops;
    double std_gflops;
    double snr;
    double chebyshev;
} dd_tune_report;

/* ---- Delay table (Eq. 1, Section II) -------------------------------------
 * Host only, needs no GPU. freq_mhz[n_chan] in any order, f_ref_mhz > 0,
 * t_samp_s > 0, dm[n_dm] >= 0 in any order. Writes shifts[n_dm][n_chan].
 * DD_ERR_ARG if a delay is negative (a channel above f_ref with DM > 0) or
 * exceeds 2^30 samples. */
dd_status dd_compute_shifts(int32_t n_chan, const double *freq_mhz, double f_ref_mhz,
                            double t_samp_s, int32_t n_dm, const double *dm,
                            int32_t *shifts);

/* ---- Plans ---------------------------------------------------------------
 * Computes the delay table (Eq. 1), sizes T_in = S + max shift (Section
 * III-A: the input holds the samples needed at the highest trial DM), builds
 * the per-tile staging tables and uploads them to the current device. The
 * plan then serves dd_execute for any input/output buffers of its shape.
 * n_out >= 1, batch >= 1. On failure *out is NULL. */
dd_status dd_plan_create(dd_plan *out, int32_t n_chan, const double *freq_mhz,
                         double f_ref_mhz, double t_samp_s, int32_t n_dm,
                         const double *dm, int64_t n_out, int32_t batch,
                         dd_dtype in_dtype);

/* Same, from an explicit non-negative delay table shifts[n_dm][n_chan]
 * (e.g. the all-zero table of the paper's DM = 0 experiment, Section IV-C). */
dd_status dd_plan_create_from_shifts(dd_plan *out, int32_t n_chan, int32_t n_dm,
                                     const int32_t *shifts, int64_t n_out,
                                     int32_t batch, dd_dtype in_dtype);

void dd_plan_destroy(dd_plan plan);

int64_t dd_plan_input_len(dd_plan plan);     /* T_in = S + max shift (elements) */
int64_t dd_plan_input_stride(dd_plan plan);  /* padded row length (elements)    */
int32_t dd_plan_max_shift(dd_plan plan);
/* Copies the delay table, int32 [n_dm][n_chan], to host memory. */
dd_status dd_plan_shifts(dd_plan plan, int32_t *host_dst);

/* Variant used by dd_execute. set: DD_ERR_ARG if the variant is not in the
 * compiled grid or does not fit the device's shared memory for this plan;
 * before it frees the old tables it waits (on the host) for this plan's
 * earlier launches on every stream they went to, not for the whole device.
 * After a launch of the plan was captured into a CUDA graph, replaced tables
 * are kept until the plan is destroyed (the graph may still replay them). */
dd_status dd_plan_get_variant(dd_plan plan, dd_variant *v);
dd_status dd_plan_set_variant(dd_plan plan, const dd_variant *v);
/* Launch order of the forward kernel's tiles: DM tiles fastest (the default;
 * resident CTAs share a time range, so windows that neighbouring DM tiles
 * share stay in L2) or time tiles fastest (resident CTAs sweep one DM tile's
 * rows; better where neighbouring DM tiles read far-apart windows, e.g. the
 * paper's LOFAR setup). dd_tune picks one for its winning variant;
 * dd_plan_set_variant resets it to DM tiles fastest. Results do not depend
 * on it. set: DD_ERR_ARG for another value. */
#define DD_ORDER_DM_FASTEST 0
#define DD_ORDER_TIME_FASTEST 1
dd_status dd_plan_get_launch_order(dd_plan plan, int32_t *order);
dd_status dd_plan_set_launch_order(dd_plan plan, int32_t order);
/* Number of compiled variants and the i-th one (0 <= i < count). */
int32_t dd_variant_count(void);
dd_status dd_variant_get(int32_t i, dd_variant *v);

/* ---- Forward (Algorithm 1; Section III-B parallelisation) ----------------
 * d_in: device [B][C][stride] of the plan's input type; d_w: device float[C]
 * (int32[C] for DD_U8); d_out: device float[B][D][S] (int32 for DD_U8).
 * Enqueues one kernel launch on `stream`; no allocation, no synchronisation. */
dd_status dd_execute(dd_plan plan, const void *d_in, const void *d_w, void *d_out,
                     void *stream);

/* The same with HOST buffers: copies h_in and h_w to plan-owned device
 * buffers (allocated on first use), runs the forward, delivers the result in
 * h_out and synchronises `stream` before returning. With pinned (page-locked)
 * buffers the output is written by the kernel straight into h_out over the
 * CPU-GPU link, and the input is pulled in up to 8 segments of whole time
 * tiles: segment s's forward launch starts as soon as the columns it needs
 * (its samples plus the max delay) are on the device, while later columns are
 * still in flight, and the first segment's low-DM tiles start once the
 * columns of their own largest delay are in (plan-owned copy and compute
 * streams, joined to `stream`).
 * Pageable buffers are staged through plan-owned device mirrors. Not safe to
 * call concurrently on one plan. */
dd_status dd_execute_host(dd_plan plan, const void *h_in, const void *h_w, void *h_out,
                          void *stream);

/* ---- Adjoint (transpose of the forward; FP32 plans only) -----------------
 * Reverse-mode derivative of the forward (not in the paper): for a cotangent
 * g = dL/dout [B][D][S],
 *   d_gin[b][c][tau] = w[c] * sum_d g[b][d][tau - shift[d][c]]
 *                      (terms with 0 <= tau - shift < S), tau < stride,
 *   d_gw[c] = sum_b sum_d sum_t g[b][d][t] * in[b][c][t + shift[d][c]].
 * d_gin [B][C][stride] and d_gw [C] are each optional (NULL = skip); d_in is
 * required when d_gw is given. The weight gradient is reduced in a fixed
 * order (deterministic). Uses plan-owned device scratch for the partial sums,
 * so concurrent dd_adjoint calls on one plan must use one stream. */
dd_status dd_adjoint(dd_plan plan, const float *d_gout, const float *d_w,
                     const float *d_in, float *d_gin, float *d_gw, void *stream);

/* ---- Weight gradient without device allocation ---------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at the moment they need the gradient
 * (a caching allocator already holding all free memory, real-time code that
 * must not take allocator locks or trigger the implicit synchronisation of
 * cudaMalloc/cudaFree, a device memory budget fixed at start-up).
 * Computes the same d_gw[c] as dd_adjoint (FP32 plans only) from d_gout
 * [B][D][S] and d_in [B][C][stride], and allocates nothing: its partial sums
 * go to one fixed 1 MiB array in the library's device image, which every GPU
 * that loads the library holds until the process exits. Limits: n_chan <=
 * 4096 (DD_ERR_ARG beyond). The first call on a device looks up that array's
 * address with the device current; make that first call before any stream
 * capture. Every call on a device shares the array and leaves its partial
 * sums there (each call overwrites all it reads), so calls that may overlap
 * on the GPU (different streams without ordering) race and must not be
 * issued. Deterministic: same inputs, same bits. */
dd_status dd_grad_w_noalloc(dd_plan plan, const float *d_gout, const float *d_in,
                            float *d_gw, void *stream);

/* ---- Auto-tuning (Section IV-A / V-A) ------------------------------------
 * Times every compiled variant that fits this plan on scratch buffers it
 * allocates and frees itself, keeps the fastest as the plan's variant and
 * fills *rep (nullable). budget_ms bounds the sweep (0 = no bound). Plans
 * whose input and output exceed 16 MB are timed with L2 flushed before each
 * timed launch; smaller ones warm (replayed back to back, their data stays
 * in L2).
 * Tuning cache: when the environment variable DD_TUNE_CACHE names a file,
 * dd_tune appends one text line "<key> kind dpt spt warps_dm warps_time
 * chans_per_stage stages order" for the winner (order: its launch order, see
 * dd_plan_set_launch_order; a line without it means DM tiles fastest), the
 * key being the device name,
 * input type, n_chan, n_dm, n_out, batch and a hash of the delay table; plan
 * creation (dd_plan_create, dd_plan_create_from_shifts) then starts from the
 * last line whose key matches, so the sweep is an offline step, as the paper
 * treats it. A missing or unreadable file, or a recorded variant that no
 * longer fits, falls back to the built-in defaults silently. */
dd_status dd_tune(dd_plan plan, int32_t budget_ms, dd_tune_report *rep);

/* Tunes the kernel variant of the adjoint's transposed dedispersion (the
 * gather runs the forward kernels with channels and trials swapped; see
 * dd_adjoint). Builds the adjoint's buffers if they do not exist yet. */
dd_status dd_tune_adjoint(dd_plan plan, int32_t budget_ms, dd_tune_report *rep);

/* The kernel variant the adjoint's transposed gather runs: read it, or pin
 * one (e.g. a variant an earlier dd_tune_adjoint reported). FP32 plans only
 * (DD_ERR_UNSUPPORTED otherwise); both build the adjoint's buffers if they
 * do not exist yet. dd_adjoint_set_variant returns DD_ERR_ARG, leaving the
 * current variant in place, if v does not fit the transposed plan; it
 * waits (on the host) for the transposed gather's own earlier launches, no
 * launch of which may still read the old tables; other work on the device
 * is not waited for. */
dd_status dd_adjoint_get_variant(dd_plan plan, dd_variant *v);
dd_status dd_adjoint_set_variant(dd_plan plan, const dd_variant *v);

/* ---- Batched uneven setups (many beams of several observation setups) ----
 * A batch groups n plans (different C, D, S, input types). dd_batch_execute
 * runs every plan's forward in ONE persistent kernel launch whose CTAs pull
 * (plan, beam, DM tile, time tile) work items from a device counter, and
 * captures that launch in a CUDA graph on first use for a given set of
 * pointers and stream (later calls with the same pointers replay it).
 * d_in[i], d_w[i], d_out[i] follow plan i's conventions. At most 16 plans;
 * they must share the input type and outlive the batch. Work items are taken
 * heaviest setup first. One launch runs one compiled kernel: all plans share
 * kind, dm_per_thread, samples_per_thread, stages and the number of trial
 * warps (warps_dm * warps_time); each plan has its own split of those warps
 * (its DM x time tile) and its own chans_per_stage. */
dd_status dd_batch_create(dd_batch *out, int32_t n, const dd_plan *plans);
dd_status dd_batch_execute(dd_batch batch, const void *const *d_in,
                           const void *const *d_w, void *const *d_out, void *stream);
/* The batch's common variant; set gives every plan that variant and rebuilds
 * the tables and graph, after waiting for the batch's own earlier launches
 * (not the whole device). */
dd_status dd_batch_get_variant(dd_batch batch, dd_variant *v);
dd_status dd_batch_set_variant(dd_batch batch, const dd_variant *v);
/* The variant plan i (index into the plans given to dd_batch_create) runs in
 * the batch. set changes only that plan's; DD_ERR_ARG, leaving every variant
 * as it was, if v does not share kind, dm_per_thread, samples_per_thread,
 * stages and warps_dm * warps_time with the other plans' or does not fit the
 * plan. Waits for the batch's own earlier launches (not the whole device). */
dd_status dd_batch_get_plan_variant(dd_batch batch, int32_t i, dd_variant *v);
dd_status dd_batch_set_plan_variant(dd_batch batch, int32_t i, const dd_variant *v);
/* Auto-tunes a batch (Section IV-A's experiment applied to one launch):
 * times the whole persistent launch for every compiled variant that fits all
 * of its plans, keeps the fastest as the common variant, then tries each
 * plan's other splits of the trial warps and chunk sizes in turn, keeping
 * those that shorten the launch (scratch buffers allocated and freed here).
 * The report (as dd_tune's) describes the common-variant sweep. */
dd_status dd_batch_tune(dd_batch batch, int32_t budget_ms, dd_tune_report *rep);
void dd_batch_destroy(dd_batch batch);

/* ---- Continuous streams (Section III-A's input of t samples, chunk by chunk)
 * A stream dedisperses a long observation in chunks of n_out samples per
 * channel with the plan's delays. Each push takes the next chunk d_chunk
 * [B][C][n_out] (rows of exactly n_out samples, the plan's input type) and
 * writes d_out [B][D][n_out]: output samples [k*n_out - M, (k+1)*n_out - M) of
 * the continuous stream, k = pushes so far, M = dd_stream_latency(s) = the
 * plan's largest delay; input samples before the stream's start count as
 * zero. The stream owns two device buffers of the plan's input shape and
 * keeps the last M input samples between pushes; pushes on one stream must be
 * ordered (same CUDA stream). The plan must outlive the stream. */
dd_status dd_stream_create(dd_stream *out, dd_plan plan);
dd_status dd_stream_push(dd_stream s, const void *d_chunk, const void *d_w, void *d_out,
                         void *stream);
dd_status dd_stream_reset(dd_stream s, void *stream);  /* back to an all-zero history */
int64_t dd_stream_latency(dd_stream s);
void dd_stream_destroy(dd_stream s);

/* ---- Diagnostics ---------------------------------------------------------- */
/* Failure-path check: enqueues one CTA that waits on a shared-memory
 * barrier nothing will complete, with a wait budget of budget_us
 * microseconds (1..2000000). When the budget runs out the kernel records
 * DD_ERR_TIMEOUT in the plan's device error word and returns, so the
 * context stays usable; dd_plan_check_device then reports it. */
dd_status dd_debug_wait_timeout(dd_plan plan, int32_t budget_us, void *stream);
/* Synchronises the device, reads and clears the plan's device error word:
 * DD_OK, DD_ERR_TIMEOUT (a bounded wait ran out) or DD_ERR_DEVICE. */
dd_status dd_plan_check_device(dd_plan plan);
const char *dd_status_str(dd_status s);
dd_status dd_get_last_error(void);              /* per thread */
const char *dd_last_error_message(void);        /* per thread */
int32_t dd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DD_H_ */
