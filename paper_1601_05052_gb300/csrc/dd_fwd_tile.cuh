// dd_fwd_tile.cuh -- the per-tile body of the forward dedispersion kernel,
// shared by the one-shot launch (dd_fwd.cu) and the persistent batched
// launch (dd_batch.cu).
//
// A tile is (beam b, DM tile of Dt trials, time tile of Ts output samples)
// and computes out[b][d][t] = sum_c w[c] * in[b][c][t + shift[d][c]] for its
// trials and samples (Algorithm 1, Section III-A, with weights; the 2-D
// work-group decomposition of Section III-B). Each warp owns DPT trials by
// 32*SPT samples; a thread accumulates DPT x SPT outputs in registers.
//
// Staging (Section III-B's shared "local memory"): for each chunk of
// channels one elected thread copies, per channel, the union of the tile's
// shifted input windows with one 1-D TMA bulk copy into a pipeline slot,
// together with the chunk's table of per-trial smem offsets. Slots are
// recycled through two mbarriers each: `full` (TMA transaction bytes) and
// `empty` (one arrival per warp once it has read the slot), so warps never
// wait for each other at a CTA-wide barrier.
//
// Two ways to turn a staged window into sums (the `kind` of a variant):
//  kind 0, lane-strided: lane l owns samples l, l+32, ...; every add reads
//    its operand from shared memory (conflict-free, one word per add).
//  kind 1, register window: a thread owns SPT consecutive samples (SPT odd
//    so that a warp's loads hit 32 distinct banks). Per channel it loads the
//    union window of its warp's DPT trials, SPT + span words, into registers
//    once and serves all DPT trials from it: the trial's delay relative to
//    the group's smallest one is warp-uniform and selects, through a switch
//    over 0..RMAX, a fully unrolled block with compile-time register indices.
//    That cuts shared-memory reads per add from 1 to (SPT+span)/(DPT*SPT).
//    Channels whose group span exceeds RMAX take the kind-0 style path.
//  kind 2, sub-band partial sums: channels form groups of 4; inside a DM
//    tile the trials of a group share only a few distinct relative delay
//    patterns, so after a chunk lands the CTA builds each pattern's weighted
//    4-channel partial series in shared memory once, and the lane-strided
//    trial loop then adds one partial value per group instead of one input
//    value per channel (the same sums, associated per group).
//  kind 3, warp-specialised sub-band: kind 2's arithmetic, but 4 extra
//    builder warps turn staged windows into partial series while the trial
//    warps consume earlier ones; full/empty mbarriers on the staging slots
//    and on 3 partial-sum slots replace every CTA-wide barrier.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "dd_ptx.cuh"

// The compiled forward kernels: X(kind, dm_per_thread, samples_per_thread).
#define DD_FWD_KEYS(X)                                                                   \
    X(0, 2, 4) X(0, 4, 2) X(0, 4, 4) X(0, 8, 2) X(0, 8, 4) X(0, 4, 8) X(1, 8, 9) X(1, 4, 15) \
        X(2, 4, 4) X(2, 4, 8) X(2, 8, 4) X(2, 8, 2) X(3, 8, 4) X(3, 4, 8) X(3, 8, 2)

namespace dd {

// Largest relative delay inside a warp's trial group served from registers.
constexpr int kRwRmax = 15;

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
    const int4 *bdesc;  // kind 2 only
    int p_elems;        // kind 2 only
    int *err;
};

// Channels per group and patterns per group of the sub-band kinds; builder
// warps and partial-sum slots of kind 3.
constexpr int kSbG = 4;
constexpr int kSbP = 8;
constexpr int kWsBuilders = 4;
constexpr int kWsPSlots = 3;

// Loads the DPT uint16 smem offsets of this warp's trials with one vector
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

// kind 0: lane-strided samples, one shared-memory read per add.
template <typename T, int DPT, int SPT>
struct LaneStrided {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    __device__ static int sample_of(int lane, int j) { return lane + 32 * j; }
    __device__ static void channel(Acc (&acc)[DPT][SPT], const T *sdata, int lane_base,
                                   const int (&o)[DPT], Wt wc) {
        const T *s = sdata + lane_base;
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            const T *src = s + o[i];
#pragma unroll
            for (int j = 0; j < SPT; ++j) acc[i][j] += wc * Elem<T>::val(src[32 * j]);
        }
    }
    __device__ static int lane_base(int wt, int lane) { return wt * 32 * SPT + lane; }
};

// kind 1: thread-contiguous samples served from a register window.
template <typename T, int DPT, int SPT>
struct RegWindow {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    static_assert(SPT % 2 == 1, "odd samples_per_thread keeps window loads conflict-free");
    static constexpr int R = kRwRmax;
    __device__ static int sample_of(int lane, int j) { return lane * SPT + j; }
    __device__ static int lane_base(int wt, int lane) { return wt * 32 * SPT + lane * SPT; }

    template <int RR>
    __device__ static __forceinline__ void add_shifted(Acc (&a)[SPT], const Acc (&win)[SPT + R],
                                                       Wt wc) {
#pragma unroll
        for (int j = 0; j < SPT; ++j) a[j] += wc * win[RR + j];
    }

    __device__ static void channel(Acc (&acc)[DPT][SPT], const T *sdata, int lane_base,
                                   const int (&o)[DPT], Wt wc) {
        int gb = o[0], gm = o[0];
#pragma unroll
        for (int i = 1; i < DPT; ++i) {
            gb = min(gb, o[i]);
            gm = max(gm, o[i]);
        }
        const int span = gm - gb;  // warp-uniform
        const T *src = sdata + lane_base + gb;
        if (span <= R) {
            Acc win[SPT + R];
#pragma unroll
            for (int k = 0; k < SPT; ++k) win[k] = Elem<T>::val(src[k]);
#pragma unroll
            for (int k = SPT; k < SPT + R; ++k) win[k] = (k < SPT + span) ? Elem<T>::val(src[k]) : Acc(0);
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                switch (o[i] - gb) {
#define DD_RW_CASE(RR) \
    case RR: add_shifted<RR>(acc[i], win, wc); break;
                    DD_RW_CASE(0) DD_RW_CASE(1) DD_RW_CASE(2) DD_RW_CASE(3) DD_RW_CASE(4)
                    DD_RW_CASE(5) DD_RW_CASE(6) DD_RW_CASE(7) DD_RW_CASE(8) DD_RW_CASE(9)
                    DD_RW_CASE(10) DD_RW_CASE(11) DD_RW_CASE(12) DD_RW_CASE(13) DD_RW_CASE(14)
                    default: add_shifted<15>(acc[i], win, wc); break;
#undef DD_RW_CASE
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const T *s = src + (o[i] - gb);
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += wc * Elem<T>::val(s[j]);
            }
        }
    }
};

template <int KIND, typename T, int DPT, int SPT>
using FwdPolicy = typename std::conditional<KIND == 1, RegWindow<T, DPT, SPT>,
                                            LaneStrided<T, DPT, SPT>>::type;

// Shared-memory layout of a forward CTA: `full` mbarriers at byte 0, `empty`
// mbarriers at byte 64 (stages <= 4), then `stages` slots of (data, offsets)
// from byte 128.
// kind 3 uses bars[4..6] / bars[12..14] for its partial-sum slots and counts
// builder warps on the staging slots' empty barriers.
template <int KIND>
__device__ __forceinline__ void fwd_init_barriers(uint64_t *bars, int stages) {
    if (threadIdx.x == 0) {
        const int n_warps = int(blockDim.x >> 5);
        const int builders = KIND == 3 ? kWsBuilders : n_warps;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&bars[8 + s], uint32_t(builders));
        }
        if (KIND == 3) {
            for (int q = 0; q < kWsPSlots; ++q) {
                mbar_init(&bars[4 + q], uint32_t(kWsBuilders));
                mbar_init(&bars[12 + q], uint32_t(n_warps - kWsBuilders));
            }
        }
        fence_barrier_init();
    }
    __syncthreads();
}

// Computes one tile. `kbase` counts the chunks this CTA has already pushed
// through its slots; chunk kg uses slot kg % stages, and the n-th completion
// of a slot's full/empty barrier belongs to chunk slot + n * stages, so the
// phase parities carry over from tile to tile without re-initialisation.
template <int KIND, typename T, int DPT, int SPT>
__device__ __forceinline__ void fwd_tile(const FwdArgs &a, int dtile, int ttile, int b,
                                         uint64_t *bars, unsigned char *stage0,
                                         uint32_t &kbase) {
    using P = FwdPolicy<KIND, T, DPT, SPT>;
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full = bars;
    uint64_t *empty = bars + 8;
    const uint32_t S = uint32_t(a.stages);
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

    // Elected thread: stage tile chunk k (global chunk kbase + k).
    auto issue = [&](int k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        if (kg >= S) mbar_wait_bounded(&empty[slot], ((kg / S) - 1u) & 1u, a.err);
        fence_proxy_async_smem();
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
        const int pro = min(int(S), n_chunks);
        for (int k = 0; k < pro; ++k) issue(k);
    }

    Acc acc[DPT][SPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = Acc(0);
    const int lb = P::lane_base(wt, lane);

    for (int k = 0; k < n_chunks; ++k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        mbar_wait_bounded(&full[slot], (kg / S) & 1u, a.err);
        const unsigned char *sb = stage0 + slot * stage_bytes;
        const T *sdata = reinterpret_cast<const T *>(sb);
        const uint16_t *soffs =
            reinterpret_cast<const uint16_t *>(sb + a.stage_data_bytes) + wd * DPT;
        const int c0 = k * a.cch;
        const int nch = min(a.cch, a.C - c0);
        for (int cc = 0; cc < nch; ++cc) {
            const Wt wc = __ldg(w + c0 + cc);
            int o[DPT];
            load_offsets<DPT>(soffs + cc * a.Dt, o);
            P::channel(acc, sdata, lb, o, wc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        // refill the slot of the previous chunk (one chunk of slack for the
        // other warps), keeping stages-1 chunks in flight
        if (tid == 0 && k >= 1 && k - 1 + int(S) < n_chunks) issue(k - 1 + int(S));
    }
    // the last chunk's slot: refills for k-1+S < n_chunks were all issued above
    kbase += uint32_t(n_chunks);

    Acc *out = static_cast<Acc *>(a.out);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = dtile * a.Dt + wd * DPT + i;
        if (d >= a.D) continue;
        Acc *orow = out + ((long long)b * a.D + d) * a.S + t0 + (lb - 0);
        const long long tmax = a.S - t0 - lb;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int off = P::sample_of(0, j);
            if (off < tmax) orow[off] = acc[i][j];
        }
    }
}


// Builds one partial series: dst[u] = sum_{j<gn} wg[j] * raw[r[j] + u] for
// u < L, lanes of a warp striding by 32 and each lane keeping 4 elements in
// flight so the shared-memory loads overlap.
template <typename T>
__device__ __forceinline__ void sb_build(typename Elem<T>::Acc *dst, const T *raw,
                                         const int (&r)[4], const typename Elem<T>::W (&wg)[4],
                                         int gn, int L, int lane) {
    using Acc = typename Elem<T>::Acc;
    if (gn == kSbG) {
        const T *r0 = raw + r[0], *r1 = raw + r[1], *r2 = raw + r[2], *r3 = raw + r[3];
        int u = lane;
        for (; u + 96 < L; u += 128) {
            Acc v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = u + 32 * q;
                v[q] = wg[0] * Elem<T>::val(r0[x]) + wg[1] * Elem<T>::val(r1[x]) +
                       wg[2] * Elem<T>::val(r2[x]) + wg[3] * Elem<T>::val(r3[x]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[u + 32 * q] = v[q];
        }
        for (; u < L; u += 32)
            dst[u] = wg[0] * Elem<T>::val(r0[u]) + wg[1] * Elem<T>::val(r1[u]) +
                     wg[2] * Elem<T>::val(r2[u]) + wg[3] * Elem<T>::val(r3[u]);
    } else {  // the last group of a plan may hold fewer channels
        for (int u = lane; u < L; u += 32) {
            Acc v = wg[0] * Elem<T>::val(raw[r[0] + u]);
#pragma unroll
            for (int j = 1; j < kSbG; ++j)
                if (j < gn) v += wg[j] * Elem<T>::val(raw[r[j] + u]);
            dst[u] = v;
        }
    }
}

// kind 2: sub-band partial sums (see the file comment). One CTA barrier per
// chunk separates the build of the chunk's partial series from the trial
// loop; the partial-sum buffer alternates between two halves by global chunk
// parity so a chunk's build never overwrites what slower warps still read.
template <typename T, int DPT, int SPT>
__device__ __forceinline__ void fwd_tile_sb(const FwdArgs &a, int dtile, int ttile, int b,
                                            uint64_t *bars, unsigned char *stage0,
                                            uint32_t &kbase) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full = bars;
    const uint32_t S = uint32_t(a.stages);
    const int stage_bytes = a.stage_data_bytes + a.stage_offs_bytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_warps = int(blockDim.x >> 5);
    const int wd = warp % a.warps_dm, wt = warp / a.warps_dm;
    const long long t0 = (long long)ttile * a.Ts;
    const T *in_b = static_cast<const T *>(a.in) + (long long)b * a.C * a.stride;
    const Wt *w = static_cast<const Wt *>(a.w);
    const int n_chunks = (a.C + a.cch - 1) / a.cch;
    const int gpc = a.cch / kSbG;
    const int g_pad = a.C_pad / kSbG;
    const int4 *desc_k = a.desc + (size_t)dtile * a.C_pad;
    const uint16_t *offs_k = a.offs + (size_t)dtile * g_pad * a.Dt;
    const int4 *bdesc_k = a.bdesc + (size_t)dtile * g_pad * kSbP * 2;
    const uint32_t poffs_bytes = uint32_t(gpc) * a.Dt * 2;
    const uint32_t bdesc_bytes = uint32_t(gpc) * kSbP * 32;
    Acc *pbuf = reinterpret_cast<Acc *>(stage0 + S * stage_bytes);

    auto issue = [&](int k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        fence_proxy_async_smem();
        unsigned char *sb = stage0 + slot * stage_bytes;
        const int c0 = k * a.cch;
        const int nch = min(a.cch, a.C - c0);
        uint32_t total = poffs_bytes + bdesc_bytes;
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
        const int g0i = c0 / kSbG;
        bulk_g2s(sb + a.stage_data_bytes, offs_k + (size_t)g0i * a.Dt, poffs_bytes, &full[slot]);
        bulk_g2s(sb + a.stage_data_bytes + poffs_bytes, bdesc_k + (size_t)g0i * kSbP * 2,
                 bdesc_bytes, &full[slot]);
    };

    if (tid == 0) {
        const int pro = min(int(S), n_chunks);
        for (int k = 0; k < pro; ++k) issue(k);
    }

    Acc acc[DPT][SPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = Acc(0);
    const int lb = wt * 32 * SPT + lane;

    for (int k = 0; k < n_chunks; ++k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        mbar_wait_bounded(&full[slot], (kg / S) & 1u, a.err);
        const unsigned char *sb = stage0 + slot * stage_bytes;
        const T *raw = reinterpret_cast<const T *>(sb);
        const uint16_t *poffs = reinterpret_cast<const uint16_t *>(sb + a.stage_data_bytes);
        const int4 *bd = reinterpret_cast<const int4 *>(sb + a.stage_data_bytes + poffs_bytes);
        Acc *P = pbuf + (kg & 1u) * a.p_elems;
        const int c0 = k * a.cch;
        const int ng = (min(a.cch, a.C - c0) + kSbG - 1) / kSbG;

        // build every pattern's partial series of this chunk
        for (int e = warp; e < ng * kSbP; e += n_warps) {
            const int4 A = bd[2 * e];
            if (A.y == 0) continue;
            const int4 B = bd[2 * e + 1];
            const int g = e / kSbP;
            const int gn = B.z;
            const int r[4] = {A.z, A.w, B.x, B.y};
            Wt wg[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) wg[j] = j < gn ? __ldg(w + c0 + g * kSbG + j) : Wt(0);
            sb_build<T>(P + A.x, raw, r, wg, gn, A.y, lane);
        }
        __syncthreads();
        // every warp has finished the trial loop of chunk k-1 (it precedes the
        // build of chunk k), so that chunk's slot, offsets included, is free
        if (tid == 0 && k >= 1 && k - 1 + int(S) < n_chunks) issue(k - 1 + int(S));

        // trial loop over the chunk's channel groups
        const Acc *Pl = P + lb;
        for (int g = 0; g < ng; ++g) {
            int o[DPT];
            load_offsets<DPT>(poffs + g * a.Dt + wd * DPT, o);
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const Acc *src = Pl + o[i];
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += src[32 * j];
            }
        }
    }
    kbase += uint32_t(n_chunks);

    Acc *out = static_cast<Acc *>(a.out);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = dtile * a.Dt + wd * DPT + i;
        if (d >= a.D) continue;
        Acc *orow = out + ((long long)b * a.D + d) * a.S + t0 + lb;
        const long long tmax = a.S - t0 - lb;
#pragma unroll
        for (int j = 0; j < SPT; ++j)
            if (32 * j < tmax) orow[32 * j] = acc[i][j];
    }
}

// kind 3: warp-specialised sub-band. Warps [0, NC) are trial warps (as in
// kind 2), warps [NC, NC + 4) builders. Barriers: full/empty of the staging
// slots at bars[0..3] / bars[8..11], full/empty of the partial-sum slots at
// bars[4..6] / bars[12..14]. A partial-sum slot holds the chunk's partial
// series followed by its per-group trial offsets (copied out of the staging
// slot so that slot can be refilled as soon as the builders are done).
template <typename T, int DPT, int SPT>
__device__ __forceinline__ void fwd_tile_ws(const FwdArgs &a, int dtile, int ttile, int b,
                                            uint64_t *bars, unsigned char *stage0,
                                            uint32_t &kbase) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full_r = bars, *empty_r = bars + 8, *full_p = bars + 4, *empty_p = bars + 12;
    const uint32_t S = uint32_t(a.stages), Q = uint32_t(kWsPSlots);
    const int stage_bytes = a.stage_data_bytes + a.stage_offs_bytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nc = int(blockDim.x >> 5) - kWsBuilders;  // trial warps
    const long long t0 = (long long)ttile * a.Ts;
    const int n_chunks = (a.C + a.cch - 1) / a.cch;
    const int gpc = a.cch / kSbG;
    const uint32_t poffs_bytes = uint32_t(gpc) * a.Dt * 2;
    const int pslot_bytes = a.p_elems * int(sizeof(Acc)) + int(poffs_bytes);
    unsigned char *pslot0 = stage0 + S * stage_bytes;

    if (warp >= nc) {
        // ---------------- builder warps
        const int bw = warp - nc;
        const T *in_b = static_cast<const T *>(a.in) + (long long)b * a.C * a.stride;
        const Wt *w = static_cast<const Wt *>(a.w);
        const int g_pad = a.C_pad / kSbG;
        const int4 *desc_k = a.desc + (size_t)dtile * a.C_pad;
        const uint16_t *offs_k = a.offs + (size_t)dtile * g_pad * a.Dt;
        const int4 *bdesc_k = a.bdesc + (size_t)dtile * g_pad * kSbP * 2;
        const uint32_t bdesc_bytes = uint32_t(gpc) * kSbP * 32;
        auto issue = [&](int k) {  // one lane of builder warp 0
            const uint32_t kg = kbase + uint32_t(k);
            const int slot = int(kg % S);
            if (kg >= S) mbar_wait_bounded(&empty_r[slot], ((kg / S) - 1u) & 1u, a.err);
            fence_proxy_async_smem();
            unsigned char *sb = stage0 + slot * stage_bytes;
            const int c0 = k * a.cch;
            const int nch = min(a.cch, a.C - c0);
            uint32_t total = poffs_bytes + bdesc_bytes;
            for (int cc = 0; cc < nch; ++cc) {
                const int4 dsc = desc_k[c0 + cc];
                const long long n = min((long long)dsc.y, a.stride - (t0 + dsc.x));
                total += uint32_t(n) * uint32_t(sizeof(T));
            }
            mbar_arrive_expect_tx(&full_r[slot], total);
            for (int cc = 0; cc < nch; ++cc) {
                const int4 dsc = desc_k[c0 + cc];
                const long long g0 = t0 + dsc.x;
                const long long n = min((long long)dsc.y, a.stride - g0);
                bulk_g2s(sb + (size_t)dsc.z * sizeof(T),
                         in_b + (long long)(c0 + cc) * a.stride + g0,
                         uint32_t(n) * uint32_t(sizeof(T)), &full_r[slot]);
            }
            const int g0i = c0 / kSbG;
            bulk_g2s(sb + a.stage_data_bytes, offs_k + (size_t)g0i * a.Dt, poffs_bytes,
                     &full_r[slot]);
            bulk_g2s(sb + a.stage_data_bytes + poffs_bytes, bdesc_k + (size_t)g0i * kSbP * 2,
                     bdesc_bytes, &full_r[slot]);
        };
        if (bw == 0 && lane == 0) {
            const int pro = min(int(S), n_chunks);
            for (int k = 0; k < pro; ++k) issue(k);
        }
        __syncwarp();
        for (int k = 0; k < n_chunks; ++k) {
            const uint32_t kg = kbase + uint32_t(k);
            const int rs = int(kg % S), ps = int(kg % Q);
            mbar_wait_bounded(&full_r[rs], (kg / S) & 1u, a.err);
            if (kg >= Q) mbar_wait_bounded(&empty_p[ps], ((kg / Q) - 1u) & 1u, a.err);
            const unsigned char *sb = stage0 + rs * stage_bytes;
            const T *raw = reinterpret_cast<const T *>(sb);
            const int4 *bd = reinterpret_cast<const int4 *>(sb + a.stage_data_bytes + poffs_bytes);
            unsigned char *pb = pslot0 + ps * pslot_bytes;
            Acc *P = reinterpret_cast<Acc *>(pb);
            const int c0 = k * a.cch;
            const int ng = (min(a.cch, a.C - c0) + kSbG - 1) / kSbG;
            for (int e = bw; e < ng * kSbP; e += kWsBuilders) {
                const int4 A = bd[2 * e];
                if (A.y == 0) continue;
                const int4 B = bd[2 * e + 1];
                const int g = e / kSbP;
                const int gn = B.z;
                Wt wg[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) wg[j] = j < gn ? __ldg(w + c0 + g * kSbG + j) : Wt(0);
                const int r[4] = {A.z, A.w, B.x, B.y};
                sb_build<T>(P + A.x, raw, r, wg, gn, A.y, lane);
            }
            if (bw == 0) {  // the trial offsets travel with the partial sums
                const uint32_t *src = reinterpret_cast<const uint32_t *>(sb + a.stage_data_bytes);
                uint32_t *dsto = reinterpret_cast<uint32_t *>(pb + a.p_elems * int(sizeof(Acc)));
                for (int i = lane; i < int(poffs_bytes / 4); i += 32) dsto[i] = src[i];
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&full_p[ps]);
                mbar_arrive(&empty_r[rs]);
            }
            // refill the staging slot of the previous chunk (one chunk of slack)
            if (bw == 0 && lane == 0 && k >= 1 && k - 1 + int(S) < n_chunks) issue(k - 1 + int(S));
            __syncwarp();
        }
        kbase += uint32_t(n_chunks);
        return;
    }

    // ---------------- trial warps
    const int wd = warp % a.warps_dm, wt = warp / a.warps_dm;
    Acc acc[DPT][SPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = Acc(0);
    const int lb = wt * 32 * SPT + lane;
    for (int k = 0; k < n_chunks; ++k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int ps = int(kg % Q);
        mbar_wait_bounded(&full_p[ps], (kg / Q) & 1u, a.err);
        const unsigned char *pb = pslot0 + ps * pslot_bytes;
        const Acc *Pl = reinterpret_cast<const Acc *>(pb) + lb;
        const uint16_t *poffs =
            reinterpret_cast<const uint16_t *>(pb + a.p_elems * int(sizeof(Acc))) + wd * DPT;
        const int c0 = k * a.cch;
        const int ng = (min(a.cch, a.C - c0) + kSbG - 1) / kSbG;
        for (int g = 0; g < ng; ++g) {
            int o[DPT];
            load_offsets<DPT>(poffs + g * a.Dt, o);
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const Acc *src = Pl + o[i];
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += src[32 * j];
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_p[ps]);
    }
    kbase += uint32_t(n_chunks);

    Acc *out = static_cast<Acc *>(a.out);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = dtile * a.Dt + wd * DPT + i;
        if (d >= a.D) continue;
        Acc *orow = out + ((long long)b * a.D + d) * a.S + t0 + lb;
        const long long tmax = a.S - t0 - lb;
#pragma unroll
        for (int j = 0; j < SPT; ++j)
            if (32 * j < tmax) orow[32 * j] = acc[i][j];
    }
}

// Dispatches a tile to the kind's body.
template <int KIND, typename T, int DPT, int SPT>
__device__ __forceinline__ void fwd_tile_any(const FwdArgs &a, int dtile, int ttile, int b,
                                             uint64_t *bars, unsigned char *stage0,
                                             uint32_t &kbase) {
    if constexpr (KIND == 2)
        fwd_tile_sb<T, DPT, SPT>(a, dtile, ttile, b, bars, stage0, kbase);
    else if constexpr (KIND == 3)
        fwd_tile_ws<T, DPT, SPT>(a, dtile, ttile, b, bars, stage0, kbase);
    else
        fwd_tile<KIND, T, DPT, SPT>(a, dtile, ttile, b, bars, stage0, kbase);
}

}  // namespace dd
