// dd_noalloc.cu -- weight gradient of the forward dedispersion that makes no
// device allocation at call time.
//
// Some callers cannot call cudaMalloc when they need this result: code that
// runs while a framework's caching allocator owns all free device memory,
// real-time pipelines that must not take the allocator's locks or its
// implicit device synchronisation, and hosts that fix their whole device
// memory budget at start-up. dd_adjoint serves grad_w through a plan-owned
// partial-sum buffer it allocates on first use; this entry point computes
// the same
//     gw[c] = sum_b sum_d sum_t g[b][d][t] * in[b][c][t + shift[d][c]]
// with its partial sums in a fixed-size array that lives in the library's
// own device image (file-scope __device__ storage), so nothing is allocated:
// the delay table is the device copy the plan made when it was created.
//
// Work split: the outputs are cut into tiles of 16 trials by 256 samples per
// beam; CTA k of G takes tiles k, k + G, ...; each warp keeps its own per-channel
// running sums in shared memory, the CTA adds its warps in a fixed order
// into row k of the scratch array, and a second kernel adds the G rows in a
// fixed order. Results are therefore reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "dd_internal.h"
#include "dd_reduce.cuh"

namespace dd {
namespace {

// Capacity of the scratch array: G rows of C floats, G * C <= this.
constexpr int kNoAllocScratchFloats = 1 << 18;  // 1 MiB per device
// Per-warp running sums live in shared memory: 8 warps * C floats.
constexpr int kNoAllocMaxChan = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

// Tiling of this kernel: 8 warps, 4 along trials and 2 along time; a thread
// covers 4 trials by 4 lane-strided samples.
constexpr int kNaDpt = 4, kNaSpt = 4, kNaWarpsDm = 4, kNaWarpsT = 2;
constexpr int kNaDt = kNaDpt * kNaWarpsDm, kNaTs = 32 * kNaSpt * kNaWarpsT;

struct NoAllocArgs {
    const float *g;       // [B][D][S]
    const float *in;      // [B][C][stride]
    const int32_t *shifts;  // [D][C]
    float *part;          // [G][C] (the scratch array)
    int C, D, B;
    long long S, stride;
    int n_dtiles, n_ttiles;
};

template <int DPT, int SPT>
__global__ void __launch_bounds__(256, 1) dd_gw_noalloc_kernel(const NoAllocArgs a) {
    extern __shared__ float wsum[];  // [n_warps][C]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_warps = blockDim.x >> 5;
    const int wd = warp % kNaWarpsDm, wt = warp / kNaWarpsDm;
    for (int e = tid; e < n_warps * a.C; e += blockDim.x) wsum[e] = 0.f;
    __syncthreads();
    float *mine = wsum + warp * a.C;

    const long long n_items = (long long)a.n_dtiles * a.n_ttiles * a.B;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int dtile = int(item % a.n_dtiles);
        const long long rest = item / a.n_dtiles;
        const int ttile = int(rest % a.n_ttiles);
        const int b = int(rest / a.n_ttiles);
        const long long tb = (long long)ttile * kNaTs + wt * 32 * SPT + lane;
        // this thread's cotangent values (zero outside the output)
        float gr[DPT][SPT];
        bool dv[DPT];
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            const int d = dtile * kNaDt + wd * DPT + i;
            dv[i] = d < a.D;
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                const long long t = tb + 32 * j;
                gr[i][j] = (dv[i] && t < a.S) ? __ldg(a.g + ((long long)b * a.D + d) * a.S + t)
                                              : 0.f;
            }
        }
        const int32_t *sh_k = a.shifts + (size_t)(dtile * kNaDt + wd * DPT) * a.C;
        for (int c = 0; c < a.C; ++c) {
            const float *row = a.in + ((long long)b * a.C + c) * a.stride;
            float p = 0.f;
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                if (!dv[i]) continue;
                const int shift = __ldg(sh_k + (size_t)i * a.C + c);
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    const long long t = tb + 32 * j;
                    if (t < a.S) p += gr[i][j] * __ldg(row + t + shift);
                }
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) p += __shfl_xor_sync(0xffffffffu, p, m);
            if (lane == 0) mine[c] += p;
        }
    }
    __syncthreads();
    for (int c = tid; c < a.C; c += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < n_warps; ++w) s += wsum[w * a.C + c];
        a.part[(long long)blockIdx.x * a.C + c] = s;
    }
}

// gw[c] = sum of the G partial rows in FP32, in a fixed order.
__global__ void dd_gw_noalloc_reduce_kernel(const float *part, int G, int C, float *gw) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    gw[c] = fixed_order_sum(part + c, G, C);
}

// Device address of the scratch array, looked up once per device (with that
// device current) on the first call made on it.
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kMaxDevices] = {};
bool g_noalloc_attr_set[kMaxDevices] = {};

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_grad_w_noalloc(dd_plan p, const float *d_gout, const float *d_in,
                                       float *d_gw, void *stream) {
    if (!p || !d_gout || !d_in || !d_gw) return fail(DD_ERR_ARG, "null argument");
    if (p->dtype != DD_F32) return fail(DD_ERR_UNSUPPORTED, "grad_w takes FP32 plans only");
    if (!aligned16(d_gout) || !aligned16(d_in) || !aligned16(d_gw))
        return fail(DD_ERR_ARG, "device pointers must be 16-byte aligned");
    if (p->C > kNoAllocMaxChan)
        return fail(DD_ERR_ARG, "dd_grad_w_noalloc supports at most 4096 channels");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(DD_ERR_ARG, "make the plan's device current first");
    if (dev < 0 || dev >= kMaxDevices) return fail(DD_ERR_UNSUPPORTED, "device index too large");
    const int block = 32 * kNaWarpsDm * kNaWarpsT;
    const size_t smem = size_t(block / 32) * p->C * sizeof(float);
    float *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
            g_noalloc_ptr[dev] = static_cast<float *>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
        if (!g_noalloc_attr_set[dev]) {
            // the largest per-warp shared-memory table any plan may need
            const int max_smem = 8 * kNoAllocMaxChan * int(sizeof(float));
            e = cudaFuncSetAttribute(dd_gw_noalloc_kernel<kNaDpt, kNaSpt>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(no-alloc)");
            g_noalloc_attr_set[dev] = true;
        }
    }
    const int n_dtiles = (p->D + kNaDt - 1) / kNaDt;
    const long long n_ttiles = (p->S + kNaTs - 1) / kNaTs;
    const long long n_items = (long long)n_dtiles * n_ttiles * p->B;
    long long G = std::min<long long>(n_items, 2LL * p->sm_count);
    G = std::min<long long>(G, kNoAllocScratchFloats / p->C);
    if (G < 1) G = 1;

    if (n_ttiles > (1LL << 30)) return fail(DD_ERR_ARG, "too many samples");
    NoAllocArgs a;
    a.g = d_gout;
    a.in = d_in;
    a.shifts = p->d_shifts;
    a.part = scratch;
    a.C = p->C;
    a.D = p->D;
    a.B = p->B;
    a.S = p->S;
    a.stride = p->stride;
    a.n_dtiles = n_dtiles;
    a.n_ttiles = int(n_ttiles);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dd_gw_noalloc_kernel<kNaDpt, kNaSpt><<<int(G), block, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dd_grad_w_noalloc launch");
    dd_gw_noalloc_reduce_kernel<<<(p->C + 127) / 128, 128, 0, st>>>(scratch, int(G), p->C, d_gw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dd_grad_w_noalloc reduce launch");
    return DD_OK;
}
