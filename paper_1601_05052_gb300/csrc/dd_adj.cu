// dd_adj.cu -- adjoint of the forward dedispersion (FP32 plans).
//
// For a cotangent g = dL/dout the input gradient is the transpose of the
// forward map. Written as a gather,
//     G[b][c][tau]   = sum_d g[b][d][tau - shift[d][c]]   (0 <= tau-shift < S)
//     gin[b][c][tau] = w[c] * G[b][c][tau]
//     gw[c]          = sum_b sum_tau in[b][c][tau] * G[b][c][tau]
// (= sum_b sum_d sum_t g[b][d][t] * in[b][c][t + shift[d][c]]).
//
// The gather is itself a dedispersion with the roles of channels and trials
// swapped: with M = the plan's largest delay rounded up to a multiple of 4
// and g' the cotangent rows padded by M zeros in front (g'[b][d][u] =
// g[b][d][u - M], zero outside [M, M+S)),
//     G[b][c][tau] = sum_d 1 * g'[b][d][tau + (M - shift[d][c])],
// i.e. the forward with D "channels", C "trials", delays M - shift >= 0 and
// unit weights, over tau < stride. So the adjoint runs the same tuned forward
// kernels (sub-band or lane-strided) on a private transposed plan. That plan
// knows that its input is zero outside columns [M, M + S): its tiles skip the
// chunks of trials whose staged windows lie wholly in the zero borders
// (about a fifth of the gather's work at 16 x 512 x 1024 x 8192). Per call:
// one copy kernel moving g into the padded buffer (its zero borders are
// written once; M is a multiple of 4 so that rows move as 16-byte words when
// S allows), one forward launch writing G into gin (or scratch), and a fused
// epilogue that scales gin by w and forms each (beam, channel)'s share of
// grad_w with a fixed-order block reduction; a last kernel adds the beams in
// FP32 in a fixed order, so results are bitwise reproducible.
#include <algorithm>
#include <vector>

#include "dd_internal.h"
#include "dd_reduce.cuh"

namespace dd {

namespace {

constexpr int kEpiThreads = 256;

// One CTA per (beam, channel) row: part[row] = sum_{tau < T_in} in * G (if
// requested) and gin[row] = w[c] * G over the padded row (if requested; G may
// alias gin).
__global__ void __launch_bounds__(kEpiThreads) dd_adj_epilogue(
    const float *G, const float *__restrict__ w, const float *__restrict__ in, float *gin,
    float *part, int C, long long stride, long long T_in) {
    const long long row = blockIdx.x;
    const int c = int(row % C);
    const float *Gr = G + row * stride;
    float s = 0.f;
    if (part) {
        const float *ir = in + row * stride;
        for (long long t = threadIdx.x; t < T_in; t += kEpiThreads) s += __ldg(ir + t) * Gr[t];
    }
    __syncthreads();  // every thread has read its G values before any is scaled in place
    if (gin) {
        const float wc = __ldg(w + c);
        float *gr = gin + row * stride;
        const float4 *G4 = reinterpret_cast<const float4 *>(Gr);
        float4 *g4 = reinterpret_cast<float4 *>(gr);
        for (long long t = threadIdx.x; t < stride / 4; t += kEpiThreads) {
            float4 v = G4[t];
            v.x *= wc;
            v.y *= wc;
            v.z *= wc;
            v.w *= wc;
            g4[t] = v;
        }
    }
    if (part) {
        __shared__ float red[kEpiThreads / 32];
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.f;
            for (int i = 0; i < kEpiThreads / 32; ++i) tot += red[i];
            part[row] = tot;
        }
    }
}

// gw[c] = sum over beams of part[b][c] in FP32, in a fixed order.
__global__ void dd_gw_reduce_kernel(const float *part, int B, int C, float *gw) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    gw[c] = fixed_order_sum(part + c, B, C);
}

// g'[row][M + t] = g[row][t] for t < S: block item i copies columns
// [i % nb * kPadCols, ...) of row i / nb; 16-byte words when both row
// starts are 16-byte aligned, single floats otherwise.
constexpr int kPadThreads = 256;
constexpr int kPadCols = 4 * 4 * kPadThreads;  // floats per block item
__global__ void __launch_bounds__(kPadThreads) dd_pad_rows_kernel(
    float *__restrict__ gpad, const float *__restrict__ g, long long S, long long pitch,
    long long M, long long nb, bool vec) {
    const long long row = blockIdx.x / nb;
    const long long c0 = (blockIdx.x % nb) * kPadCols;
    const float *src = g + row * S;
    float *dst = gpad + row * pitch + M;
    if (vec) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long c = c0 / 4 + threadIdx.x + k * kPadThreads;
            if (c < S / 4) d4[c] = s4[c];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const long long c = c0 + threadIdx.x + k * kPadThreads;
            if (c < S) dst[c] = src[c];
        }
    }
}

__global__ void dd_fill_kernel(float *p, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

void free_adj_state(AdjState *a) {
    if (a->plan) dd_plan_destroy(a->plan);
    if (a->gpad) cudaFree(a->gpad);
    if (a->ones) cudaFree(a->ones);
    if (a->part) cudaFree(a->part);
    if (a->gscr) cudaFree(a->gscr);
    *a = AdjState{};
}

// Builds the transposed plan and its buffers on first use.
dd_status ensure_adj_state(dd_plan_s *p) {
    if (p->adj.plan) return DD_OK;
    AdjState a;
    a.M = (p->max_shift + 3) / 4 * 4;
    std::vector<int32_t> sh(size_t(p->C) * p->D);
    for (int d = 0; d < p->D; ++d)
        for (int c = 0; c < p->C; ++c)
            sh[size_t(c) * p->D + d] = a.M - p->shifts[size_t(d) * p->C + c];
    dd_status s =
        dd_plan_create_from_shifts(&a.plan, p->D, p->C, sh.data(), p->stride, p->B, DD_F32);
    if (s != DD_OK) return s;
    // the padded cotangent is zero outside columns [M, M + S) of each row:
    // the transposed plan's tables skip chunks that would only add zeros
    a.plan->nz_lo = a.M;
    a.plan->nz_hi = a.M + p->S;
    {
        const dd_variant v0 = a.plan->fwd.v;
        s = dd_plan_set_variant(a.plan, &v0);
        if (s != DD_OK) {
            dd_plan_destroy(a.plan);
            return s;
        }
    }
    const dd_plan_s *q = a.plan;
    const size_t gpad_elems = size_t(p->B) * p->D * q->stride;
    cudaError_t e = cudaMalloc(&a.gpad, gpad_elems * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(a.gpad, 0, gpad_elems * sizeof(float), q->aux);
    if (e == cudaSuccess) e = cudaMalloc(&a.ones, size_t(p->D) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&a.part, size_t(p->B) * p->C * sizeof(float));
    if (e == cudaSuccess) {
        dd_fill_kernel<<<(p->D + 255) / 256, 256, 0, q->aux>>>(a.ones, p->D, 1.0f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->aux);  // only the set-up work
    if (e != cudaSuccess) {
        free_adj_state(&a);
        return cuda_fail(e, "adjoint buffers");
    }
    p->adj = a;
    return DD_OK;
}

dd_status launch_adjoint(dd_plan_s *p, const float *g, const float *w, const float *in,
                         float *gin, float *gw, cudaStream_t st) {
    AdjState &a = p->adj;
    dd_plan_s *q = a.plan;
    float *G = gin;
    if (!G) {  // grad_w only: G goes to scratch
        if (!a.gscr) {
            cudaError_t e =
                cudaMalloc(&a.gscr, size_t(p->B) * p->C * p->stride * sizeof(float));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(adjoint scratch)");
        }
        G = a.gscr;
    }
    // g'[b][d][M + t] = g[b][d][t]; the zero borders were written at allocation
    const long long rows = (long long)p->B * p->D;
    const long long nb = (p->S + kPadCols - 1) / kPadCols;
    const bool vec = p->S % 4 == 0 && a.M % 4 == 0 && q->stride % 4 == 0;
    dd_pad_rows_kernel<<<unsigned(rows * nb), kPadThreads, 0, st>>>(a.gpad, g, p->S, q->stride,
                                                                     a.M, nb, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "padded cotangent copy");
    dd_status s = launch_forward(q, q->fwd, a.gpad, a.ones, G, st);
    if (s != DD_OK) return s;
    dd_adj_epilogue<<<unsigned(size_t(p->B) * p->C), kEpiThreads, 0, st>>>(
        G, w, in, gin, gw ? a.part : nullptr, p->C, p->stride, p->T_in);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint epilogue launch");
    if (gw) {
        dd_gw_reduce_kernel<<<(p->C + 127) / 128, 128, 0, st>>>(a.part, p->B, p->C, gw);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "grad_w reduce launch");
    }
    return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_tune_adjoint(dd_plan p, int32_t budget_ms, dd_tune_report *rep) {
    if (!p) return fail(DD_ERR_ARG, "null plan");
    if (p->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "the adjoint takes FP32 plans only");
    {
        std::lock_guard<std::mutex> lk(p->mu);
        dd_status s = ensure_adj_state(p);
        if (s != DD_OK) return s;
    }
    return dd_tune(p->adj.plan, budget_ms, rep);
}

extern "C" dd_status dd_adjoint_get_variant(dd_plan p, dd_variant *v) {
    if (!p || !v) return fail(DD_ERR_ARG, "null argument");
    if (p->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "the adjoint takes FP32 plans only");
    std::lock_guard<std::mutex> lk(p->mu);
    dd_status s = ensure_adj_state(p);
    if (s != DD_OK) return s;
    return dd_plan_get_variant(p->adj.plan, v);
}

extern "C" dd_status dd_adjoint_set_variant(dd_plan p, const dd_variant *v) {
    if (!p || !v) return fail(DD_ERR_ARG, "null argument");
    if (p->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "the adjoint takes FP32 plans only");
    std::lock_guard<std::mutex> lk(p->mu);
    dd_status s = ensure_adj_state(p);
    if (s != DD_OK) return s;
    return dd_plan_set_variant(p->adj.plan, v);
}

extern "C" dd_status dd_adjoint(dd_plan p, const float *d_gout, const float *d_w,
                                const float *d_in, float *d_gin, float *d_gw, void *stream) {
    if (!p || !d_gout) return fail(DD_ERR_ARG, "null argument");
    if (p->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "the adjoint takes FP32 plans only");
    if (!d_gin && !d_gw) return DD_OK;
    if (d_gin && !d_w) return fail(DD_ERR_ARG, "d_w is required for d_gin");
    if (d_gw && !d_in) return fail(DD_ERR_ARG, "d_in is required for d_gw");
    const void *ptrs[] = {d_gout, d_w, d_in, d_gin, d_gw};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return fail(DD_ERR_ARG, "device pointers must be 16-byte aligned");
    std::lock_guard<std::mutex> lk(p->mu);
    dd_status s = ensure_adj_state(p);
    if (s != DD_OK) return s;
    return launch_adjoint(p, d_gout, d_w, d_in, d_gin, d_gw, static_cast<cudaStream_t>(stream));
}
