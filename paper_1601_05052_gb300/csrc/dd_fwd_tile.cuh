// dd_fwd_tile.cuh -- the per-tile body of the forward dedispersion kernel,
// shared by the one-shot launch (dd_fwd.cu) and the persistent batched
// launch (dd_batch.cu).
//
// A tile is (beam b, DM tile of Dt trials, time tile of Ts output samples)
// and computes out[b][d][t] = sum_c w[c] * in[b][c][t + shift[d][c]] for its
// trials and samples (Algorithm 1, Section III-A, with weights; 2-D
// work-group decomposition of Section III-B). A thread accumulates DPT
// trials by SPT samples in registers; lanes own consecutive samples (sample
// t = lane + 32 j of the warp's range) so shared-memory reads are
// conflict-free and global stores coalesced. For each chunk of channels one
// elected thread copies, per channel, the union of the tile's shifted input
// windows (Section III-B's shared "local memory" staging) with one 1-D TMA
// bulk copy into a pipeline slot; the chunk's table of per-trial smem
// offsets rides along in the same slot.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "dd_ptx.cuh"

// The compiled (dm_per_thread, samples_per_thread) grid of forward kernels.
#define DD_FWD_KEYS(X) X(2, 4) X(4, 2) X(4, 4) X(8, 2) X(8, 4) X(4, 8)

namespace dd {

template <typename T>
struct Elem;
template <>
struct Elem<float> {
    using Acc = float;
    using W = float;
    __device__ static float val(float x) { return x; }
};
template <>
struct Elem<__half> {
    using Acc = float;
    using W = float;
    __device__ static float val(__half x) { return __half2float(x); }
};
template <>
struct Elem<__nv_bfloat16> {
    using Acc = float;
    using W = float;
    __device__ static float val(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <>
struct Elem<uint8_t> {
    using Acc = int;
    using W = int;
    __device__ static int val(uint8_t x) { return int(x); }
};

// Everything a tile needs about one plan and one set of buffers.
struct FwdArgs {
    const void *in;
    const void *w;
    void *out;
    int C, D;
    long long S, stride;
    int Dt, Ts, C_pad, cch, stages, warps_dm;
    int stage_data_bytes, stage_offs_bytes;
    int n_dtiles, n_ttiles, B;
    const int4 *desc;
    const uint16_t *offs;
    int *err;
};

// Loads the DPT uint16 smem offsets of this thread's trials with one vector
// load (4/8/16-byte aligned by construction of the tables).
template <int DPT>
__device__ __forceinline__ void load_offsets(const uint16_t *p, int (&o)[DPT]) {
    if constexpr (DPT == 8) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = int(w[i] & 0xffffu);
            o[2 * i + 1] = int(w[i] >> 16);
        }
    } else if constexpr (DPT == 4) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        o[0] = int(v.x & 0xffffu);
        o[1] = int(v.x >> 16);
        o[2] = int(v.y & 0xffffu);
        o[3] = int(v.y >> 16);
    } else {
        static_assert(DPT == 2, "DPT must be 2, 4 or 8");
        const uint32_t v = *reinterpret_cast<const uint32_t *>(p);
        o[0] = int(v & 0xffffu);
        o[1] = int(v >> 16);
    }
}

// Computes one tile. `full` holds a.stages mbarriers; `kbase` counts the
// chunks this CTA has already consumed through them (so the phase parity of
// every slot carries over from tile to tile without re-initialisation). On
// return no copy is in flight and every thread is past a CTA barrier.
template <typename T, int DPT, int SPT>
__device__ __forceinline__ void fwd_tile(const FwdArgs &a, int dtile, int ttile, int b,
                                         uint64_t *full, unsigned char *stage0,
                                         uint32_t &kbase) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    const int stage_bytes = a.stage_data_bytes + a.stage_offs_bytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wd = warp % a.warps_dm, wt = warp / a.warps_dm;
    const long long t0 = (long long)ttile * a.Ts;
    const T *in_b = static_cast<const T *>(a.in) + (long long)b * a.C * a.stride;
    const Wt *w = static_cast<const Wt *>(a.w);
    const int n_chunks = (a.C + a.cch - 1) / a.cch;
    const int4 *desc_k = a.desc + (size_t)dtile * a.C_pad;
    const uint16_t *offs_k = a.offs + (size_t)dtile * a.C_pad * a.Dt;
    const uint32_t offs_bytes = uint32_t(a.cch) * a.Dt * 2;

    auto issue = [&](int k) {
        const int slot = int((kbase + uint32_t(k)) % uint32_t(a.stages));
        unsigned char *sb = stage0 + slot * stage_bytes;
        const int c0 = k * a.cch;
        const int nch = min(a.cch, a.C - c0);
        uint32_t total = offs_bytes;
        for (int cc = 0; cc < nch; ++cc) {
            const int4 dsc = desc_k[c0 + cc];
            const long long n = min((long long)dsc.y, a.stride - (t0 + dsc.x));
            total += uint32_t(n) * uint32_t(sizeof(T));
        }
        mbar_arrive_expect_tx(&full[slot], total);
        for (int cc = 0; cc < nch; ++cc) {
            const int4 dsc = desc_k[c0 + cc];
            const long long g0 = t0 + dsc.x;
            const long long n = min((long long)dsc.y, a.stride - g0);
            bulk_g2s(sb + (size_t)dsc.z * sizeof(T), in_b + (long long)(c0 + cc) * a.stride + g0,
                     uint32_t(n) * uint32_t(sizeof(T)), &full[slot]);
        }
        bulk_g2s(sb + a.stage_data_bytes, offs_k + (size_t)c0 * a.Dt, offs_bytes, &full[slot]);
    };

    if (tid == 0) {
        fence_proxy_async_smem();
        const int pro = min(a.stages - 1, n_chunks);
        for (int k = 0; k < pro; ++k) issue(k);
    }

    Acc acc[DPT][SPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = Acc(0);

    for (int k = 0; k < n_chunks; ++k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % uint32_t(a.stages));
        if (tid == 0 && k + a.stages - 1 < n_chunks) {
            fence_proxy_async_smem();
            issue(k + a.stages - 1);
        }
        mbar_wait_bounded(&full[slot], (kg / uint32_t(a.stages)) & 1u, a.err);
        const unsigned char *sb = stage0 + slot * stage_bytes;
        const T *sdata = reinterpret_cast<const T *>(sb) + wt * 32 * SPT + lane;
        const uint16_t *soffs =
            reinterpret_cast<const uint16_t *>(sb + a.stage_data_bytes) + wd * DPT;
        const int c0 = k * a.cch;
        const int nch = min(a.cch, a.C - c0);
        for (int cc = 0; cc < nch; ++cc) {
            const Wt wc = __ldg(w + c0 + cc);
            int o[DPT];
            load_offsets<DPT>(soffs + cc * a.Dt, o);
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const T *src = sdata + o[i];
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += wc * Elem<T>::val(src[32 * j]);
            }
        }
        __syncthreads();
    }
    kbase += uint32_t(n_chunks);

    Acc *out = static_cast<Acc *>(a.out);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = dtile * a.Dt + wd * DPT + i;
        if (d >= a.D) continue;
        Acc *orow = out + ((long long)b * a.D + d) * a.S;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const long long t = t0 + wt * 32 * SPT + lane + 32 * j;
            if (t < a.S) orow[t] = acc[i][j];
        }
    }
}

// Shared-memory layout of a forward CTA: stage mbarriers in the first 128
// bytes, then `stages` slots of (data, offsets).
__device__ __forceinline__ void fwd_init_barriers(uint64_t *full, int stages) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
}

}  // namespace dd
