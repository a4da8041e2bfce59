// dd_fwd.cu -- forward dedispersion kernel for sm_103a and its launcher.
//
// Computes out[b][d][t] = sum_c w[c] * in[b][c][t + shift[d][c]] (Algorithm
// 1, Section III-A, with weights) with one CTA per (DM tile, time tile,
// beam); the tile body is in dd_fwd_tile.cuh. By default the DM tile runs
// fastest along grid x, so that CTAs resident at the same time share time
// ranges and the input windows they stage stay in L2. Where neighbouring DM
// tiles read far-apart windows (delays that grow by more than a time tile
// per trial), the tuner can take the time tile fastest instead: resident
// CTAs then sweep one DM tile's rows, and the next DM tile, whose windows
// are shifted by a few DM steps, finds them still in L2.
#include <algorithm>
#include <atomic>
#include <limits>

#include "dd_fwd_tile.cuh"
#include "dd_internal.h"

namespace dd {

// LIVE: the plan has a live-chunk table (the adjoint's transposed gather,
// FP32 only); tiles sum only their live chunks.
template <int KIND, typename T, int DPT, int SPT, bool LIVE>
__global__ void __launch_bounds__(fwd_max_threads(KIND), fwd_min_blocks(KIND, DPT, SPT))
    dd_fwd_kernel(const FwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    fwd_init_barriers<KIND>(bars, a.stages);
    uint32_t kbase = 0;
    const int x = int(blockIdx.x);
    const int dt = a.time_major ? x / a.grid_tt : x % a.grid_dt;
    const int tt = a.time_major ? x % a.grid_tt : x / a.grid_dt;
    fwd_tile_any<KIND, T, DPT, SPT, LIVE>(a, a.dtile0 + dt, a.ttile0 + tt, blockIdx.y, bars,
                                          smem + 128, kbase);
}

// One CTA waits on an mbarrier that nothing arrives at, bounded by budget_ns.
__global__ void dd_wait_timeout_kernel(int *err, unsigned long long budget_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0u, err, budget_ns);
}

// Copies n 16-byte words with all SMs (used to pull pinned host memory over
// the CPU-GPU link at the link's rate rather than one copy engine's).
__global__ void dd_copy16_kernel(uint4 *__restrict__ dst, const uint4 *__restrict__ src,
                                 size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x)
        dst[i] = src[i];
}

// Copies columns [w0, w1) (16-byte words) of `rows` rows of `pitch` words
// with all SMs.
__global__ void dd_copy_cols16_kernel(uint4 *__restrict__ dst, const uint4 *__restrict__ src,
                                      size_t rows, size_t pitch, size_t w0, size_t w1) {
    const size_t width = w1 - w0, n = rows * width;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        const size_t r = i / width, c = w0 + i % width;
        dst[r * pitch + c] = src[r * pitch + c];
    }
}

// Device-side address of a page-locked host buffer, or null for pageable or
// device memory.
const void *mapped_host_ptr(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return at.devicePointer;
}
void *mapped_host_ptr(void *p) { return const_cast<void *>(mapped_host_ptr(static_cast<const void *>(p))); }

namespace {

using FwdLaunchFn = cudaError_t (*)(const FwdArgs &, dim3, dim3, size_t, cudaStream_t);

constexpr int kMaxDevices = 64;

template <int KIND, typename T, int DPT, int SPT, bool LIVE>
cudaError_t launch_fwd_t(const FwdArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    // Make sure the kernel's dynamic shared-memory limit (set per device)
    // covers smem, checking once per size increase; the limit is only ever
    // raised, since other launches of the same kernel may need more.
    static std::atomic<size_t> smem_set[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kMaxDevices;
    if (smem > 48 * 1024 && (!cached || smem > smem_set[dev].load())) {
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, dd_fwd_kernel<KIND, T, DPT, SPT, LIVE>);
        if (e != cudaSuccess) return e;
        if (size_t(fa.maxDynamicSharedSizeBytes) < smem) {
            e = cudaFuncSetAttribute(dd_fwd_kernel<KIND, T, DPT, SPT, LIVE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
        }
        if (cached) smem_set[dev].store(smem);
    }
    dd_fwd_kernel<KIND, T, DPT, SPT, LIVE><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, bool LIVE>
FwdLaunchFn pick(int kind, int dpt, int spt) {
#define DD_PICK(K_, D_, S_) \
    if (kind == K_ && dpt == D_ && spt == S_) return &launch_fwd_t<K_, T, D_, S_, LIVE>;
    DD_FWD_KEYS(DD_PICK)
#undef DD_PICK
    return nullptr;
}

// Live-chunk kernels exist for FP32 only (the adjoint's transposed gather).
FwdLaunchFn pick_fn(dd_dtype t, int kind, int dpt, int spt, bool live) {
    if (live) return t == DD_F32 ? pick<float, true>(kind, dpt, spt) : nullptr;
    switch (t) {
        case DD_F32: return pick<float, false>(kind, dpt, spt);
        case DD_F16: return pick<__half, false>(kind, dpt, spt);
        case DD_BF16: return pick<__nv_bfloat16, false>(kind, dpt, spt);
        case DD_U8: return pick<uint8_t, false>(kind, dpt, spt);
    }
    return nullptr;
}

template <typename T, bool LIVE>
const void *pick_kernel(int kind, int dpt, int spt) {
#define DD_PICK_K(K_, D_, S_) \
    if (kind == K_ && dpt == D_ && spt == S_) return (const void *)&dd_fwd_kernel<K_, T, D_, S_, LIVE>;
    DD_FWD_KEYS(DD_PICK_K)
#undef DD_PICK_K
    return nullptr;
}

}  // namespace

int fwd_resident_per_sm(const dd_plan_s *p, const FwdTables &t) {
    const int kind = t.v.kind, dpt = t.v.dm_per_thread, spt = t.v.samples_per_thread;
    const void *k = nullptr;
    if (t.d_live)
        k = p->dtype == DD_F32 ? pick_kernel<float, true>(kind, dpt, spt) : nullptr;
    else if (p->dtype == DD_F32)
        k = pick_kernel<float, false>(kind, dpt, spt);
    else if (p->dtype == DD_F16)
        k = pick_kernel<__half, false>(kind, dpt, spt);
    else if (p->dtype == DD_BF16)
        k = pick_kernel<__nv_bfloat16, false>(kind, dpt, spt);
    else
        k = pick_kernel<uint8_t, false>(kind, dpt, spt);
    if (!k) return 0;
    const int block = 32 * (t.v.warps_dm * t.v.warps_time + extra_warps(kind));
    // the query needs the kernel's dynamic shared-memory limit at least this
    // large; like launch_fwd_t, it only ever raises it
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (size_t(fa.maxDynamicSharedSizeBytes) < t.smem_bytes &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t.smem_bytes)) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, t.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

const std::vector<FwdKernelKey> &fwd_compiled_keys() {
    static const std::vector<FwdKernelKey> keys = {
#define DD_KEY(K_, D_, S_) FwdKernelKey{K_, D_, S_},
        DD_FWD_KEYS(DD_KEY)
#undef DD_KEY
    };
    return keys;
}

bool fwd_variant_compiled(int kind, int dpt, int spt) {
    return pick_fn(DD_F32, kind, dpt, spt, false) != nullptr;
}

dd_status launch_forward(dd_plan_s *p, const FwdTables &t, const void *in, const void *w,
                         void *out, cudaStream_t st, int ttile0, int n_ttiles, int dtile0,
                         int n_dtiles) {
    if (n_ttiles < 0) n_ttiles = t.n_ttiles - ttile0;
    if (ttile0 < 0 || n_ttiles <= 0 || ttile0 + n_ttiles > t.n_ttiles)
        return fail(DD_ERR_ARG, "time-tile range");
    if (n_dtiles < 0) n_dtiles = t.n_dtiles - dtile0;
    if (dtile0 < 0 || n_dtiles <= 0 || dtile0 + n_dtiles > t.n_dtiles)
        return fail(DD_ERR_ARG, "DM-tile range");
    FwdLaunchFn fn = pick_fn(p->dtype, t.v.kind, t.v.dm_per_thread, t.v.samples_per_thread,
                             t.d_live != nullptr);
    if (!fn) return fail(DD_ERR_UNSUPPORTED, "forward variant not compiled");
    FwdArgs a;
    a.in = in;
    a.w = w;
    a.out = out;
    a.C = p->C;
    a.D = p->D;
    a.S = p->S;
    a.stride = p->stride;
    a.Dt = t.Dt;
    a.Ts = t.Ts;
    a.C_pad = t.C_pad;
    a.cch = t.v.chans_per_stage;
    a.stages = t.v.stages;
    a.warps_dm = t.v.warps_dm;
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
    a.p_elems = t.p_elems;
    a.live = t.d_live;
    a.err = p->d_err;
    a.ttile0 = ttile0;
    a.dtile0 = dtile0;
    a.grid_tt = n_ttiles;
    a.grid_dt = n_dtiles;
    a.time_major = t.time_major ? 1 : 0;
    if ((long long)n_dtiles * n_ttiles > 0x7fffffffLL) return fail(DD_ERR_ARG, "too many tiles");
    dim3 grid(unsigned(n_dtiles * n_ttiles), unsigned(p->B));
    dim3 block(unsigned(32 * (t.v.warps_dm * t.v.warps_time + extra_warps(t.v.kind))));
    cudaError_t e = fn(a, grid, block, t.smem_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    p->launches.note(st);
    return DD_OK;
}

// dd_execute_host with a pinned input: the input is pulled in segments of
// whole time tiles, and segment s's forward launch starts as soon as its
// columns are on the device. Segment s needs columns [0, min(T_in, end of its
// last time tile + max shift)) of every row; each segment copies only the
// columns beyond the previous one's, so the input crosses the link once. The
// first increment (at least max shift columns) is pulled by an SM copy kernel
// at the link's rate, in two parts. The first part holds the columns of the
// first launch: a prefix of DM tiles (delays grow with DM) over the
// segment's first time tiles, the rectangle that needs the fewest columns
// among those with at least as many tiles as the launch's last partial round
// of resident CTAs (q below). The SMs that run one tile more than the others
// set the end of the call, so only an earlier start for them shortens it.
// Later increments go by the copy engine, leaving the SMs to the forward
// launches, which alternate between two streams so one segment's last wave
// overlaps the next segment's first.
dd_status host_pipeline(dd_plan_s *p, const void *in_dev, const void *h_in, const void *h_w,
                        void *out, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        if (!p->hx_stream[i]) e = cudaStreamCreateWithFlags(&p->hx_stream[i], cudaStreamNonBlocking);
    for (int i = 0; i < kHostSegments + 5 && e == cudaSuccess; ++i)
        if (!p->hx_event[i]) e = cudaEventCreateWithFlags(&p->hx_event[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
    cudaStream_t cs = p->hx_stream[0];
    cudaEvent_t *ev = p->hx_event;
    cudaEvent_t ev_start = ev[kHostSegments], ev_c1 = ev[kHostSegments + 1],
                ev_c2 = ev[kHostSegments + 2], ev_low = ev[kHostSegments + 3],
                ev_c3 = ev[kHostSegments + 4];
    const FwdTables &t = p->fwd;
    const size_t elt = size_t(elt_bytes(p->dtype));
    const size_t pitch_w = size_t(p->stride) * elt / 16;  // row pitch in 16-byte words
    const size_t rows = size_t(p->B) * p->C;
    const int nseg = std::min(kHostSegments, t.n_ttiles);
    const int per = (t.n_ttiles + nseg - 1) / nseg;
    // all streams start after the work already queued on the caller's stream
    e = cudaEventRecord(ev_start, st);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(p->hx_stream[i], ev_start, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->h_w_dev, h_w, size_t(p->C) * 4, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline start");
    size_t w_done = 0;
    auto words = [&](long long cols) {
        return std::min(pitch_w, (size_t(std::min<long long>(p->T_in, cols)) * elt + 15) / 16);
    };
    for (int sgi = 0, tt = 0; tt < t.n_ttiles; ++sgi, tt += per) {
        const int n_t = std::min(per, t.n_ttiles - tt);
        const long long t_end = std::min<long long>(p->S, (long long)(tt + n_t) * t.Ts);
        const long long cols = std::min<long long>(p->T_in, t_end + p->max_shift);
        const size_t w_need = words(cols);
        if (sgi == 0) {
            // the first launch: DM tiles [0, k1) x time tiles [0, n1) (see above)
            const long long slots = (long long)std::max(1, fwd_resident_per_sm(p, t)) *
                                    std::max(1, p->sm_count);
            const long long total = (long long)t.n_dtiles * t.n_ttiles * p->B;
            const long long q = (total - 1) % slots + 1;
            int k1 = 0, n1 = 0;
            long long best = std::numeric_limits<long long>::max();
            int32_t run = 0;
            for (int k = 1; k < t.n_dtiles; ++k) {
                run = std::max(run, t.dtile_max_shift[size_t(k - 1)]);
                // the fewest time tiles that give this prefix q tiles
                const long long n = (q + (long long)k * p->B - 1) / ((long long)k * p->B);
                if (n > n_t) continue;
                const long long c = std::min<long long>(p->S, n * t.Ts) + run;
                if (c < best) {
                    best = c;
                    k1 = k;
                    n1 = int(n);
                }
            }
            const size_t w_low = k1 ? words(best) : w_need;
            if (k1 > 0 && w_low < w_need) {
                dd_copy_cols16_kernel<<<4 * p->sm_count, 256, 0, cs>>>(
                    static_cast<uint4 *>(p->h_in_dev), static_cast<const uint4 *>(in_dev), rows,
                    pitch_w, 0, w_low);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaEventRecord(ev_low, cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hx_stream[3], ev_low, 0);
                if (e != cudaSuccess) return cuda_fail(e, "first input columns");
                dd_status s = launch_forward(p, t, p->h_in_dev, p->h_w_dev, out, p->hx_stream[3],
                                             tt, n1, 0, k1);
                if (s != DD_OK) return s;
                dd_copy_cols16_kernel<<<4 * p->sm_count, 256, 0, cs>>>(
                    static_cast<uint4 *>(p->h_in_dev), static_cast<const uint4 *>(in_dev), rows,
                    pitch_w, w_low, w_need);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaEventRecord(ev[0], cs);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hx_stream[1], ev[0], 0);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hx_stream[2], ev[0], 0);
                if (e != cudaSuccess) return cuda_fail(e, "first input segment");
                w_done = w_need;
                // the rest of the segment: the other DM tiles over the first n1 time
                // tiles, and every DM tile over the segment's remaining time tiles
                if (k1 < t.n_dtiles) {
                    s = launch_forward(p, t, p->h_in_dev, p->h_w_dev, out, p->hx_stream[1], tt, n1,
                                       k1, t.n_dtiles - k1);
                    if (s != DD_OK) return s;
                }
                if (n1 < n_t) {
                    s = launch_forward(p, t, p->h_in_dev, p->h_w_dev, out, p->hx_stream[2],
                                       tt + n1, n_t - n1);
                    if (s != DD_OK) return s;
                }
                continue;
            }
        }
        if (w_need > w_done) {
            if (sgi == 0) {
                dd_copy_cols16_kernel<<<4 * p->sm_count, 256, 0, cs>>>(
                    static_cast<uint4 *>(p->h_in_dev), static_cast<const uint4 *>(in_dev), rows,
                    pitch_w, w_done, w_need);
                e = cudaGetLastError();
            } else {
                const size_t off = w_done * 16;
                e = cudaMemcpy2DAsync(static_cast<unsigned char *>(p->h_in_dev) + off, pitch_w * 16,
                                      static_cast<const unsigned char *>(h_in) + off, pitch_w * 16,
                                      (w_need - w_done) * 16, rows, cudaMemcpyHostToDevice, cs);
            }
            if (e != cudaSuccess) return cuda_fail(e, "input segment copy");
            w_done = w_need;
        }
        cudaStream_t ks = p->hx_stream[1 + (sgi & 1)];
        e = cudaEventRecord(ev[sgi], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, ev[sgi], 0);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline event");
        dd_status s = launch_forward(p, t, p->h_in_dev, p->h_w_dev, out, ks, tt, n_t);
        if (s != DD_OK) return s;
    }
    // the caller's stream waits for every compute stream
    e = cudaEventRecord(ev_c1, p->hx_stream[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev_c2, p->hx_stream[2]);
    if (e == cudaSuccess) e = cudaEventRecord(ev_c3, p->hx_stream[3]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_c1, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_c2, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_c3, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline join");
    return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_execute(dd_plan p, const void *d_in, const void *d_w, void *d_out, void *stream) {
    if (!p || !d_in || !d_w || !d_out) return fail(DD_ERR_ARG, "null argument");
    if (!aligned16(d_in) || !aligned16(d_w) || !aligned16(d_out))
        return fail(DD_ERR_ARG, "device pointers must be 16-byte aligned");
    return launch_forward(p, p->fwd, d_in, d_w, d_out, static_cast<cudaStream_t>(stream));
}

dd_status dd_debug_wait_timeout(dd_plan p, int32_t budget_us, void *stream) {
    if (!p || budget_us < 1 || budget_us > 2000000) return fail(DD_ERR_ARG, "bad argument");
    dd_wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        p->d_err, (unsigned long long)budget_us * 1000ull);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "timeout probe launch");
    return DD_OK;
}

dd_status dd_execute_host(dd_plan p, const void *h_in, const void *h_w, void *h_out,
                          void *stream) {
    if (!p || !h_in || !h_w || !h_out) return fail(DD_ERR_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t in_bytes = size_t(p->B) * p->C * p->stride * elt_bytes(p->dtype);
    const size_t w_bytes = size_t(p->C) * 4;
    const size_t out_bytes = size_t(p->B) * p->D * p->S * 4;
    // Pinned (page-locked, mapped) host buffers are reachable from the GPU over
    // the CPU-GPU link: the input is pulled by an SM copy kernel and the
    // forward kernel writes its output straight into host memory, so no
    // output copy follows it. Pageable buffers go through device mirrors.
    const void *in_dev = mapped_host_ptr(h_in);
    void *out_dev = mapped_host_ptr(h_out);
    {
        std::lock_guard<std::mutex> lk(p->mu);
        cudaError_t e = cudaSuccess;
        if (!p->h_in_dev) e = cudaMalloc(&p->h_in_dev, in_bytes);
        if (e == cudaSuccess && !p->h_w_dev) e = cudaMalloc(&p->h_w_dev, w_bytes);
        if (e == cudaSuccess && !out_dev && !p->h_out_dev) e = cudaMalloc(&p->h_out_dev, out_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(host mirrors)");
    }
    cudaError_t e = cudaSuccess;
    void *out = out_dev ? out_dev : p->h_out_dev;
    if (in_dev && aligned16(in_dev)) {
        dd_status s = host_pipeline(p, in_dev, h_in, h_w, out, st);
        if (s != DD_OK) return s;
    } else {
        e = cudaMemcpyAsync(p->h_in_dev, h_in, in_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->h_w_dev, h_w, w_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "input upload");
        dd_status s = launch_forward(p, p->fwd, p->h_in_dev, p->h_w_dev, out, st);
        if (s != DD_OK) return s;
    }
    if (!out_dev) e = cudaMemcpyAsync(h_out, p->h_out_dev, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "output download / sync");
    return DD_OK;
}

}  // extern "C"
