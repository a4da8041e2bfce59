// dd_adj.cu -- adjoint of the forward dedispersion (FP32 plans).
//
// For a cotangent g = dL/dout the input gradient is the transpose of the
// forward map, written as a gather so that every output element is owned by
// one thread (no atomics):
//     G[b][c][tau]   = sum_d g[b][d][tau - shift[d][c]]   (0 <= tau-shift < S)
//     gin[b][c][tau] = w[c] * G[b][c][tau]
// and the weight gradient reuses the same inner sums:
//     gw[c] = sum_b sum_tau in[b][c][tau] * G[b][c][tau]
// (= sum_b sum_d sum_t g[b][d][t] * in[b][c][t + shift[d][c]]).
//
// The gather is the forward kernel's structure with the roles of channels
// and trial DMs swapped: a CTA owns Ct channels by Tt input samples and
// stages, for a chunk of trials, each trial's cotangent window covering the
// tile's channels into shared memory (zero outside [0, S)). grad_w partial
// sums per (time tile, beam, channel) go to plan-owned scratch and a second
// kernel adds them in a fixed order, so results are bitwise reproducible.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "dd_internal.h"
#include "dd_ptx.cuh"

namespace dd {

namespace {

constexpr int kAdjCpt = 4;   // channels per thread
constexpr int kAdjSpt = 4;   // samples per thread
constexpr int kAdjWc = 4;    // warps along channels
constexpr int kAdjWt = 2;    // warps along time
constexpr int kAdjDch = 16;  // trials staged per chunk

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct AdjArgs {
    const float *g, *w, *in;
    float *gin, *part;
    int C, D, B;
    long long S, T_in, stride;
    int Ct, Tt, D_pad, dch, wc, stage_elems;
    const int4 *desc;
    const uint16_t *offs;
};

template <int CPT, int SPT>
__global__ void __launch_bounds__(256, 1) dd_adj_kernel(const AdjArgs a) {
    extern __shared__ __align__(16) float sg[];
    uint16_t *soffs = reinterpret_cast<uint16_t *>(sg + a.stage_elems);
    __shared__ float red[8][32];  // [time warp][channel in tile]

    const int ctile = blockIdx.x, ttile = blockIdx.y, b = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int wcw = warp % a.wc, wt = warp / a.wc;
    const long long tau0 = (long long)ttile * a.Tt;
    const float *g_b = a.g + (long long)b * a.D * a.S;
    const int4 *desc_k = a.desc + (size_t)ctile * a.D_pad;
    const uint16_t *offs_k = a.offs + (size_t)ctile * a.D_pad * a.Ct;

    float acc[CPT][SPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = 0.f;

    for (int d0 = 0; d0 < a.D; d0 += a.dch) {
        const int nd = min(a.dch, a.D - d0);
        // cooperative, zero-filled staging of each trial's cotangent window
        for (int dd = warp; dd < nd; dd += nwarps) {
            const int4 dsc = desc_k[d0 + dd];
            const float *grow = g_b + (long long)(d0 + dd) * a.S;
            const long long ts = tau0 - dsc.x;
            for (int e = lane; e < dsc.y; e += 32) {
                const long long t = ts + e;
                sg[dsc.z + e] = (t >= 0 && t < a.S) ? __ldg(grow + t) : 0.f;
            }
        }
        for (int e = tid; e < a.dch * a.Ct; e += blockDim.x)
            soffs[e] = offs_k[(size_t)d0 * a.Ct + e];
        __syncthreads();
        const float *sbase = sg + wt * 32 * SPT + lane;
        for (int dd = 0; dd < nd; ++dd) {
            const uint16_t *op = soffs + dd * a.Ct + wcw * CPT;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const float *src = sbase + op[i];
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += src[32 * j];
            }
        }
        __syncthreads();
    }

    // epilogue: gin = w * G, and this tile's share of grad_w
    float pw[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = ctile * a.Ct + wcw * CPT + i;
        pw[i] = 0.f;
        if (c >= a.C) continue;
        const float wv = a.w ? __ldg(a.w + c) : 0.f;
        const long long row = ((long long)b * a.C + c) * a.stride;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const long long tau = tau0 + wt * 32 * SPT + lane + 32 * j;
            if (tau < a.stride && a.gin) a.gin[row + tau] = wv * acc[i][j];
            if (a.part && tau < a.T_in) pw[i] += __ldg(a.in + row + tau) * acc[i][j];
        }
    }
    if (a.part) {
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            float v = pw[i];
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
            pw[i] = v;
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < CPT; ++i) red[wt][wcw * CPT + i] = pw[i];
        }
        __syncthreads();
        const int nwt = nwarps / a.wc;
        if (tid < a.Ct) {
            const int c = ctile * a.Ct + tid;
            if (c < a.C) {
                float s = 0.f;
                for (int q = 0; q < nwt; ++q) s += red[q][tid];
                a.part[((long long)ttile * a.B + b) * a.C + c] = s;
            }
        }
    }
}

// gw[c] = sum over (time tile, beam) partials, in a fixed order, in FP64.
__global__ void dd_gw_reduce_kernel(const float *part, int n_rows, int C, float *gw) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double s = 0.0;
    for (int r = 0; r < n_rows; ++r) s += double(part[(long long)r * C + c]);
    gw[c] = float(s);
}

void free_adj_tables(AdjTables *t) {
    if (t->d_desc) cudaFree(t->d_desc);
    if (t->d_offs) cudaFree(t->d_offs);
    if (t->d_part) cudaFree(t->d_part);
    t->d_desc = nullptr;
    t->d_offs = nullptr;
    t->d_part = nullptr;
}

dd_status ensure_adj_tables(dd_plan_s *p) {
    if (p->adj.d_desc) return DD_OK;
    AdjTables t;
    t.cpt = kAdjCpt;
    t.spt = kAdjSpt;
    t.wc = kAdjWc;
    t.wt = kAdjWt;
    t.dch = kAdjDch;
    t.Ct = t.cpt * t.wc;
    t.Tt = 32 * t.spt * t.wt;
    t.n_ctiles = (p->C + t.Ct - 1) / t.Ct;
    t.n_ttiles = int((p->stride + t.Tt - 1) / t.Tt);
    t.D_pad = int(rup(p->D, t.dch));
    if (t.n_ttiles > 65535) return fail(DD_ERR_UNSUPPORTED, "input too long for the adjoint grid");
    std::vector<int4> desc(size_t(t.n_ctiles) * t.D_pad, make_int4(0, 0, 0, 0));
    std::vector<uint16_t> offs(size_t(t.n_ctiles) * t.D_pad * t.Ct, 0);
    int64_t stage_max = 0;
    for (int k = 0; k < t.n_ctiles; ++k) {
        const int c0 = k * t.Ct, c1 = std::min(p->C, c0 + t.Ct);
        for (int d0 = 0; d0 < p->D; d0 += t.dch) {
            int64_t soff = 0;
            for (int d = d0; d < std::min(p->D, d0 + t.dch); ++d) {
                int32_t smin = INT32_MAX, smax = 0;
                for (int c = c0; c < c1; ++c) {
                    const int32_t s = p->shifts[size_t(d) * p->C + c];
                    smin = std::min(smin, s);
                    smax = std::max(smax, s);
                }
                const int64_t A = rup(smax, 4);
                const int64_t len = rup(A - smin + t.Tt, 4);
                if (soff + len > 65536) return fail(DD_ERR_UNSUPPORTED, "adjoint stage too large");
                desc[size_t(k) * t.D_pad + d] = make_int4(int(A), int(len), int(soff), 0);
                for (int j = 0; j < t.Ct; ++j) {
                    const int c = c0 + j;
                    const int64_t o = c < p->C ? soff + A - p->shifts[size_t(d) * p->C + c] : soff;
                    offs[(size_t(k) * t.D_pad + d) * t.Ct + j] = uint16_t(o);
                }
                soff += len;
            }
            stage_max = std::max(stage_max, soff);
        }
    }
    t.stage_elems = int(rup(stage_max, 4));
    t.smem_bytes = size_t(t.stage_elems) * 4 + size_t(t.dch) * t.Ct * 2;
    if (t.smem_bytes > p->smem_optin) return fail(DD_ERR_UNSUPPORTED, "adjoint stage too large");
    cudaError_t e = cudaMalloc(&t.d_desc, desc.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&t.d_offs, offs.size() * sizeof(uint16_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&t.d_part, size_t(t.n_ttiles) * p->B * p->C * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(t.d_desc, desc.data(), desc.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t.d_offs, offs.data(), offs.size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_adj_tables(&t);
        return cuda_fail(e, "adjoint tables");
    }
    p->adj = t;
    return DD_OK;
}

dd_status launch_adjoint(dd_plan_s *p, const float *g, const float *w, const float *in,
                         float *gin, float *gw, cudaStream_t st) {
    const AdjTables &t = p->adj;
    AdjArgs a;
    a.g = g;
    a.w = w;
    a.in = in;
    a.gin = gin;
    a.part = gw ? t.d_part : nullptr;
    a.C = p->C;
    a.D = p->D;
    a.B = p->B;
    a.S = p->S;
    a.T_in = p->T_in;
    a.stride = p->stride;
    a.Ct = t.Ct;
    a.Tt = t.Tt;
    a.D_pad = t.D_pad;
    a.dch = t.dch;
    a.wc = t.wc;
    a.stage_elems = t.stage_elems;
    a.desc = t.d_desc;
    a.offs = t.d_offs;
    static size_t smem_set = 0;
    if (t.smem_bytes > 48 * 1024 && t.smem_bytes > smem_set) {
        cudaError_t e = cudaFuncSetAttribute(dd_adj_kernel<kAdjCpt, kAdjSpt>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(t.smem_bytes));
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(adjoint)");
        smem_set = t.smem_bytes;
    }
    dim3 grid(unsigned(t.n_ctiles), unsigned(t.n_ttiles), unsigned(p->B));
    dim3 block(unsigned(32 * t.wc * t.wt));
    dd_adj_kernel<kAdjCpt, kAdjSpt><<<grid, block, t.smem_bytes, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    if (gw) {
        dd_gw_reduce_kernel<<<(p->C + 127) / 128, 128, 0, st>>>(t.d_part, t.n_ttiles * p->B, p->C,
                                                                  gw);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "grad_w reduce launch");
    }
    return DD_OK;
}

}  // namespace dd

using namespace dd;

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
    dd_status s = ensure_adj_tables(p);
    if (s != DD_OK) return s;
    return launch_adjoint(p, d_gout, d_w, d_in, d_gin, d_gw, static_cast<cudaStream_t>(stream));
}
