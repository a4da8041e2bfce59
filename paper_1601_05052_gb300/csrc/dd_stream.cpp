// dd_stream.cpp -- continuous dedispersion of a long observation in chunks.
//
// The paper dedisperses one second of data per call with an input of t
// samples, t covering the delay at the highest trial DM (Section III-A). For
// a continuous stream the same holds chunk by chunk: chunk k of S new samples
// per channel, preceded by the previous M = max-delay samples, is exactly one
// plan input of T_in = S + M samples, and gives the S output samples
// [kS - M, (k+1)S - M) of the continuous stream (samples before the stream's
// start count as zeros). The stream keeps two device buffers in the plan's
// input layout and alternates between them: the new chunk goes behind the
// history, the forward runs, and the last M samples are copied to the head of
// the other buffer for the next chunk (two buffers, so no copy overlaps
// itself).
#include <cstring>

#include "dd_internal.h"

struct dd_stream_s {
    dd_plan plan = nullptr;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t pushed = 0;
};

using namespace dd;

extern "C" {

dd_status dd_stream_create(dd_stream *out, dd_plan plan) {
    if (!out || !plan) return fail(DD_ERR_ARG, "null argument");
    *out = nullptr;
    auto *s = new (std::nothrow) dd_stream_s;
    if (!s) return fail(DD_ERR_NOMEM, "host allocation");
    s->plan = plan;
    const size_t bytes = size_t(plan->B) * plan->C * plan->stride * elt_bytes(plan->dtype);
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMalloc(&s->buf[i], bytes);
        if (e == cudaSuccess) e = cudaMemset(s->buf[i], 0, bytes);
        if (e != cudaSuccess) {
            dd_stream_destroy(s);
            return cuda_fail(e, "stream buffers");
        }
    }
    *out = s;
    return DD_OK;
}

dd_status dd_stream_reset(dd_stream s, void *stream) {
    if (!s) return fail(DD_ERR_ARG, "null stream");
    const dd_plan p = s->plan;
    const size_t bytes = size_t(p->B) * p->C * p->stride * elt_bytes(p->dtype);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMemsetAsync(s->buf[i], 0, bytes, st);
        if (e != cudaSuccess) return cuda_fail(e, "stream reset");
    }
    s->cur = 0;
    s->pushed = 0;
    return DD_OK;
}

dd_status dd_stream_push(dd_stream s, const void *d_chunk, const void *d_w, void *d_out,
                         void *stream) {
    if (!s || !d_chunk || !d_w || !d_out) return fail(DD_ERR_ARG, "null argument");
    if (!aligned16(d_w) || !aligned16(d_out))
        return fail(DD_ERR_ARG, "device pointers must be 16-byte aligned");
    const dd_plan p = s->plan;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t elt = size_t(elt_bytes(p->dtype));
    const size_t pitch = size_t(p->stride) * elt;
    const size_t M = size_t(p->max_shift);
    unsigned char *cur = static_cast<unsigned char *>(s->buf[s->cur]);
    unsigned char *nxt = static_cast<unsigned char *>(s->buf[1 - s->cur]);
    const size_t rows = size_t(p->B) * p->C;
    // new samples behind the history: cur[row][M, M + S) = chunk[row][0, S)
    cudaError_t e = cudaMemcpy2DAsync(cur + M * elt, pitch, d_chunk, size_t(p->S) * elt,
                                      size_t(p->S) * elt, rows, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "stream chunk copy");
    dd_status r = launch_forward(p, p->fwd, cur, d_w, d_out, st);
    if (r != DD_OK) return r;
    // history for the next chunk: nxt[row][0, M) = cur[row][S, S + M)
    if (M > 0) {
        e = cudaMemcpy2DAsync(nxt, pitch, cur + size_t(p->S) * elt, pitch, M * elt, rows,
                              cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "stream history copy");
    }
    s->cur = 1 - s->cur;
    s->pushed += 1;
    return DD_OK;
}

int64_t dd_stream_latency(dd_stream s) { return s ? int64_t(s->plan->max_shift) : -1; }

void dd_stream_destroy(dd_stream s) {
    if (!s) return;
    for (int i = 0; i < 2; ++i)
        if (s->buf[i]) cudaFree(s->buf[i]);
    delete s;
}

}  // extern "C"
