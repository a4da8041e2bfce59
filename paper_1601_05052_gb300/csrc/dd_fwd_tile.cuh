// dd_fwd_tile.cuh -- the per-tile body of the forward dedispersion kernel,
// shared by the one-shot launch (dd_fwd.cu) and the persistent batched
// launch (dd_batch.cu).
//
// A tile is (beam b, DM tile of Dt trials, time tile of Ts output samples)
// and computes out[b][d][t] = sum_c w[c] * in[b][c][t + shift[d][c]] for its
// trials and samples (Algorithm 1, Section III-A, with weights; the 2-D
// work-group decomposition of Section III-B). Each trial warp owns DPT
// trials by 32*SPT samples; a thread accumulates DPT x SPT outputs in
// registers.
//
// Staging (Section III-B's shared "local memory"): channels are taken in
// chunks. For each chunk one warp copies, per channel (one lane each), the
// union of the tile's shifted input windows with a 1-D TMA bulk copy into a
// pipeline slot, together with the chunk's tables and weights; the slot's
// `full` mbarrier counts the bytes. Channel descriptors are read one chunk
// ahead so the copies go out without waiting on global memory.
//
// Ways to turn a staged window into sums (the `kind` of a variant):
//  kind 0, lane-strided: lane l owns samples l, l+32, ...; every add reads
//    its operand from shared memory (conflict-free, one word per add).
//    Slots are recycled through `empty` mbarriers (one arrival per warp).
//  kind 1, register window: a thread owns SPT (odd) consecutive samples;
//    per channel it loads its warp's union window into registers once and
//    serves every trial from it through a warp-uniform switch on the
//    trial's relative delay (0..15); wider groups take a direct path.
//  kind 2, sub-band partial sums: channels form groups of 4; inside a DM
//    tile the trials of a group share few distinct relative delay patterns,
//    so the CTA builds each pattern's weighted 4-channel partial series in
//    shared memory once per chunk and the lane-strided trial loop adds one
//    partial value per group instead of one input value per channel (the
//    same sums, associated per group). A dedicated producer warp stages the
//    chunks; the compute warps meet at one named barrier per chunk.
//  kind 4, wide sub-band: kind 2 in CTAs of up to 16 trial warps (one
//    resident CTA per SM), for DM tiles of 128 trials.
//  kind 3, warp-specialised sub-band: kind 2's arithmetic with 4 extra
//    builder warps; mbarriers on the staging slots and on 3 partial-sum
//    slots replace every CTA-wide barrier.
//  kind 5, lane-strided with shared delays: kind 0, but a trial whose delay
//    in the channel equals the previous trial's reuses the operands already
//    in registers.
//  kind 6, one-slot wide sub-band: kind 4 with a single partial-sum slot
//    (one more barrier per chunk) and up to 8 groups per chunk, so that
//    FP32 input fits 32-channel chunks.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "dd_kinds.h"
#include "dd_ptx.cuh"

// The compiled forward kernels: X(kind, dm_per_thread, samples_per_thread).
// Kind 4 is kind 2 in CTAs of up to 16 trial warps (one CTA per SM), so a
// DM tile can span 128 trials and amortise each partial series over more of them.
#define DD_FWD_KEYS(X)                                                                    \
    X(0, 2, 4) X(0, 4, 2) X(0, 4, 4) X(0, 8, 2) X(0, 8, 4) X(0, 4, 8) X(1, 8, 9) X(2, 4, 4) \
        X(2, 4, 8) X(2, 8, 4) X(2, 8, 2) X(3, 8, 4) X(3, 4, 8) X(3, 8, 2) X(4, 8, 4) X(4, 4, 8) \
            X(5, 4, 8) X(5, 8, 4) X(6, 4, 8) X(0, 4, 16)

namespace dd {

// Largest relative delay inside a warp's trial group served from registers.
constexpr int kRwRmax = 15;
// Channels per group and patterns per group of the sub-band kinds; builder
// warps and partial-sum slots of kind 3.
constexpr int kSbG = 4;
constexpr int kSbP = 8;
constexpr int kWsPSlots = 3;
// Chunks whose channel descriptors a producer warp holds in registers ahead
// of issuing their copies.
constexpr int kDescAhead = 4;

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
    // One-shot launches cover DM tiles [dtile0, dtile0 + grid_dt) by time
    // tiles [ttile0, ttile0 + grid_tt); CTA x of the launch takes them with
    // the DM tile fastest (time_major 0) or the time tile fastest (1).
    int ttile0, dtile0, grid_tt, grid_dt, time_major;
    const int4 *copies;  // staging copies [n_dtiles][n_chunks][n_copies]
    int n_copies;
    const uint16_t *offs;
    const int4 *bdesc;  // sub-band kinds: build blocks [n_dtiles][n_chunks][n_blocks]
    int n_blocks;       // sub-band kinds
    int p_elems;        // sub-band kinds
    // [n_dtiles][n_ttiles] {first, end} range of the chunks whose staged
    // windows reach the input's nonzero columns, for plans that declare zero
    // input borders (the adjoint's transposed gather); chunks outside it only
    // add zeros. Read only by kernels compiled with LIVE; null otherwise.
    const int2 *live;
    int *err;
};

// The chunks a tile stages and sums: all of them, or (kernels compiled with
// LIVE, launched for plans that have a live table) the live range.
template <bool LIVE>
__device__ __forceinline__ int2 chunk_range(const FwdArgs &a, int dtile, int ttile) {
    if constexpr (LIVE) return a.live[(size_t)dtile * a.n_ttiles + ttile];
    return make_int2(0, (a.C + a.cch - 1) / a.cch);
}

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

// Barrier over the first n threads of the CTA (named barrier 1): the
// compute warps of a kind-2 CTA synchronise without the producer warp.
__device__ __forceinline__ void compute_barrier(int n) {
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}

// Packed FP32 pair arithmetic of sm_100-class GPUs (one instruction for two
// lanes' worth of adds / fmas, each rounded to nearest like the scalar
// forms): a += b and d = a * b + d element-wise.
__device__ __forceinline__ void add2(float &a0, float &a1, float b0, float b1) {
    const float2 r = __fadd2_rn(make_float2(a0, a1), make_float2(b0, b1));
    a0 = r.x;
    a1 = r.y;
}
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(b0, b1), make_float2(d0, d1));
    d0 = r.x;
    d1 = r.y;
}

// ------------------------------------------------------------------ staging

// Per-tile staging context. Layout of a slot: [window data: stage_data_bytes]
// [tables: tab_bytes][weights: 16-byte rounded cch words].
template <typename T>
struct Stager {
    const FwdArgs &a;
    const T *in_b;
    long long t0;
    const int4 *copies_k;  // this DM tile's staging copies
    const void *tab_k;    // kind 0/1: trial offsets; sub-band kinds: group offsets
    const int4 *bdesc_k;  // sub-band kinds: this DM tile's build blocks
    uint32_t tab_bytes;   // per chunk, both tables
    uint32_t tab1_bytes;  // per chunk, first table
    unsigned char *stage0;
    int stage_bytes;
    bool subband;
    int kc0;  // chunk k of the tile's loop is chunk kc0 + k of the plan

    // This lane's first staging copy of chunk k (copy `lane`; zero if none).
    __device__ __forceinline__ int4 desc(int k, int lane) const {
        return lane < a.n_copies ? copies_k[(size_t)(kc0 + k) * a.n_copies + lane]
                                 : make_int4(0, 0, 0, 0);
    }

    // Bytes copy d moves (a window may reach past the row's padded end only
    // in the last time tile; it is cut there, on a 16-byte boundary).
    __device__ __forceinline__ uint32_t copy_bytes(int4 d) const {
        return d.y ? uint32_t(min((long long)d.y, a.stride - (t0 + d.x))) * uint32_t(sizeof(T))
                   : 0u;
    }

    __device__ __forceinline__ void copy(unsigned char *sb, int c0, int4 d, uint64_t *full) const {
        const uint32_t bytes = copy_bytes(d);
        if (bytes)
            bulk_g2s(sb + (size_t)d.z * sizeof(T),
                     in_b + (long long)(c0 + d.w) * a.stride + t0 + d.x, bytes, full);
    }

    // Warp-cooperative: stage chunk k into `slot`. Lane l issues the chunk's
    // copy l (at most 32 per chunk; `dsc` preloaded), lane 0 also the tables
    // and weights. All 32 lanes of one warp must call it.
    __device__ __forceinline__ void issue(int k, int slot, int4 dsc, uint64_t *full,
                                          int lane) const {
        unsigned char *sb = stage0 + slot * stage_bytes;
        const int c0 = (kc0 + k) * a.cch;
        const int nch = min(a.cch, a.C - c0);
        uint32_t total = copy_bytes(dsc);
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) total += __shfl_xor_sync(0xffffffffu, total, m);
        const uint32_t w_bytes = uint32_t((nch * 4 + 15) & ~15);
        if (lane == 0) mbar_arrive_expect_tx(full, total + tab_bytes + w_bytes);
        __syncwarp();
        fence_proxy_async_smem();
        copy(sb, c0, dsc, full);
        if (lane == 0) {
            unsigned char *tb = sb + a.stage_data_bytes;
            if (!subband) {
                bulk_g2s(tb, static_cast<const uint16_t *>(tab_k) + (size_t)c0 * a.Dt, tab_bytes,
                         full);
            } else {
                const int g0i = c0 / kSbG;
                bulk_g2s(tb, static_cast<const uint16_t *>(tab_k) + (size_t)g0i * a.Dt,
                         tab1_bytes, full);
                bulk_g2s(tb + tab1_bytes, bdesc_k + (size_t)(kc0 + k) * a.n_blocks,
                         tab_bytes - tab1_bytes, full);
            }
            // the chunk's weights; a 16-byte granule never crosses a page, so
            // rounding the last chunk up stays inside the weight buffer's page
            bulk_g2s(tb + tab_bytes, static_cast<const uint32_t *>(a.w) + c0, w_bytes, full);
        }
    }
};

template <typename T>
__device__ __forceinline__ Stager<T> make_stager(const FwdArgs &a, int dtile, int b, long long t0,
                                                 unsigned char *stage0, bool subband, int kc0) {
    const int gpc = a.cch / kSbG;
    const int g_pad = a.C_pad / kSbG;
    Stager<T> s{a,
                static_cast<const T *>(a.in) + (long long)b * a.C * a.stride,
                t0,
                a.copies + (size_t)dtile * ((a.C + a.cch - 1) / a.cch) * a.n_copies,
                subband ? static_cast<const void *>(a.offs + (size_t)dtile * g_pad * a.Dt)
                        : static_cast<const void *>(a.offs + (size_t)dtile * a.C_pad * a.Dt),
                subband ? a.bdesc + (size_t)dtile * ((a.C + a.cch - 1) / a.cch) * a.n_blocks
                        : nullptr,
                subband ? uint32_t(gpc) * a.Dt * 2 + uint32_t(a.n_blocks) * 16
                        : uint32_t(a.cch) * a.Dt * 2,
                subband ? uint32_t(gpc) * a.Dt * 2 : uint32_t(a.cch) * a.Dt * 2,
                stage0,
                a.stage_data_bytes + a.stage_offs_bytes,
                subband,
                kc0};
    return s;
}

// Stores a thread's accumulators (lane-strided sample mapping).
template <typename Acc, int DPT, int SPT>
__device__ __forceinline__ void store_lane_strided(const FwdArgs &a, const Acc (&acc)[DPT][SPT],
                                                   int dtile, int b, long long t0, int wd, int lb) {
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

// ------------------------------------------------------------------ kinds 0 and 1

// kind 0: lane-strided samples, one shared-memory read per add. kind 5
// (REUSE): the same, but a trial whose delay in the channel equals the
// previous trial's adds the operands already loaded for it; adjacent trials
// often share a channel's delay at low DMs and high frequencies, so this
// saves shared-memory reads there (it is a separate kernel because the test
// and branch slow down setups where no trials share a delay).
template <typename T, int DPT, int SPT, bool REUSE = false>
struct LaneStrided {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    __device__ static int sample_of(int j) { return 32 * j; }
    __device__ static int lane_base(int wt, int lane) { return wt * 32 * SPT + lane; }
    __device__ static void channel(Acc (&acc)[DPT][SPT], const T *sdata, int lane_base,
                                   const int (&o)[DPT], Wt wc) {
        const T *s = sdata + lane_base;
        if constexpr (REUSE) {
            Acc v[SPT];
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                if (i == 0 || o[i] != o[i - 1]) {
                    const T *src = s + o[i];
#pragma unroll
                    for (int j = 0; j < SPT; ++j) v[j] = Elem<T>::val(src[32 * j]);
                }
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += wc * v[j];
            }
        } else {
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const T *src = s + o[i];
#pragma unroll
                for (int j = 0; j < SPT; ++j) acc[i][j] += wc * Elem<T>::val(src[32 * j]);
            }
        }
    }
};

// kind 1: thread-contiguous samples served from a register window.
template <typename T, int DPT, int SPT>
struct RegWindow {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    static_assert(SPT % 2 == 1, "odd samples_per_thread keeps window loads conflict-free");
    static constexpr int R = kRwRmax;
    __device__ static int sample_of(int j) { return j; }
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
            for (int k = SPT; k < SPT + R; ++k)
                win[k] = (k < SPT + span) ? Elem<T>::val(src[k]) : Acc(0);
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

// Barriers: every kind uses full[s] = bars[s] (producer arrival + bytes) and
// empty[s] = bars[8 + s]: one arrival per warp for kinds 0/1, one per chunk
// for kind 2 (after its compute barrier), one per builder warp for kind 3,
// which also uses
// bars[4..6] / bars[12..14] for its partial-sum slots and counts builder
// warps on the staging slots' empty barriers.
template <int KIND>
__device__ __forceinline__ void fwd_init_barriers(uint64_t *bars, int stages) {
    if (threadIdx.x == 0) {
        const int n_warps = int(blockDim.x >> 5);
        const int releasers = KIND == 3 ? kWsBuilders : (is_subband(KIND) ? 1 : n_warps);
        for (int s = 0; s < stages; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&bars[8 + s], uint32_t(releasers));
        }
        *reinterpret_cast<volatile int *>(&bars[7]) = 0;  // the CTA's give-up flag
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

// Kinds 0, 1 and 5. `kbase` counts the chunks this CTA has already pushed
// through its slots; chunk kg uses slot kg % stages, and the n-th completion
// of a slot's full/empty barrier belongs to chunk slot + n * stages, so the
// phase parities carry over from tile to tile without re-initialisation.
template <int KIND, typename T, int DPT, int SPT, bool LIVE>
__device__ __forceinline__ void fwd_tile(const FwdArgs &a, int dtile, int ttile, int b,
                                         uint64_t *bars, unsigned char *stage0,
                                         uint32_t &kbase) {
    using P = typename std::conditional<
        KIND == 1, RegWindow<T, DPT, SPT>, LaneStrided<T, DPT, SPT, KIND == 5>>::type;
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full = bars;
    uint64_t *empty = bars + 8;
    volatile int *gave_up = reinterpret_cast<volatile int *>(&bars[7]);
    const uint32_t S = uint32_t(a.stages);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wd = warp % a.warps_dm, wt = warp / a.warps_dm;
    const long long t0 = (long long)ttile * a.Ts;
    const int2 kr = chunk_range<LIVE>(a, dtile, ttile);
    const int n_chunks = kr.y - kr.x;
    const Stager<T> st = make_stager<T>(a, dtile, b, t0, stage0, false, kr.x);

    // warp 0 stages chunk k, after the slot's previous chunk was released;
    // once a wait of the CTA has given up it issues nothing more
    auto issue = [&](int k, int4 dsc) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        bool ok = true;
        if (kg >= S)
            ok = mbar_wait_bounded(&empty[slot], ((kg / S) - 1u) & 1u, a.err, kWaitBudgetNs,
                                   gave_up);
        if (__all_sync(0xffffffffu, ok)) st.issue(k, slot, dsc, &full[slot], lane);
    };
    if (warp == 0) {
        const int pro = min(int(S), n_chunks);
        for (int k = 0; k < pro; ++k) issue(k, st.desc(k, lane));
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
        const int kn = k - 1 + int(S);  // the chunk warp 0 stages after this one
        int4 pre = make_int4(0, 0, 0, 0);
        if (warp == 0 && k >= 1 && kn < n_chunks) pre = st.desc(kn, lane);
        // A failed wait (or one that finds the CTA's give-up flag set) ends
        // the tile: the slot may hold a stale chunk, so nothing more is
        // summed, released or stored.
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], (kg / S) & 1u, a.err,
                                                       kWaitBudgetNs, gave_up)))
            break;
        const unsigned char *sb = stage0 + slot * st.stage_bytes;
        const T *sdata = reinterpret_cast<const T *>(sb);
        const uint16_t *soffs =
            reinterpret_cast<const uint16_t *>(sb + a.stage_data_bytes) + wd * DPT;
        const Wt *sw = reinterpret_cast<const Wt *>(sb + a.stage_data_bytes + st.tab_bytes);
        const int nch = min(a.cch, a.C - (kr.x + k) * a.cch);
        for (int cc = 0; cc < nch; ++cc) {
            int o[DPT];
            load_offsets<DPT>(soffs + cc * a.Dt, o);
            P::channel(acc, sdata, lb, o, sw[cc]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        // refill the slot of the previous chunk (one chunk of slack for the
        // other warps), keeping stages-1 chunks in flight
        if (warp == 0 && k >= 1 && kn < n_chunks) issue(kn, pre);
    }
    kbase += uint32_t(n_chunks);
    if (*gave_up) return;

    Acc *out = static_cast<Acc *>(a.out);
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int d = dtile * a.Dt + wd * DPT + i;
        if (d >= a.D) continue;
        Acc *orow = out + ((long long)b * a.D + d) * a.S + t0 + lb;
        const long long tmax = a.S - t0 - lb;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int off = P::sample_of(j);
            if (off < tmax) orow[off] = acc[i][j];
        }
    }
}

// ------------------------------------------------------------------ kinds 2 and 3

// Builds this worker's share of a chunk's partial series from the chunk's
// build blocks. A block covers up to 4 sub-blocks of 32 consecutive
// elements of one series: {dst, r0, (r1-r0) | (r2-r0) << 16, (r3-r0) |
// group << 16 | channels << 20 | sub-blocks << 24}, and lane l of sub-block s
// writes P[dst + 32 s + l] = sum_{j < channels} w[4 group + j] *
// raw[r_j + 32 s + l]. Worker `part` of `parts` takes blocks part, part +
// parts, ...; the next block's descriptor is loaded while the current one is
// built, and all of a block's operand loads are issued before its
// arithmetic. Blocks with 0 sub-blocks are capacity padding; they sit after
// every real block of the chunk, so a worker stops at its first one.
template <typename T>
__device__ __forceinline__ void sb_build_blocks(typename Elem<T>::Acc *P, const T *raw,
                                                const int4 *blk, const typename Elem<T>::W *sw,
                                                int n_blocks, int part, int parts, int lane) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    static_assert(sizeof(Wt) == 4, "weights are 4-byte words");
    int b = part;
    int4 d = b < n_blocks ? blk[b] : make_int4(0, 0, 0, 0);
    while (b < n_blocks) {
        const int bn = b + parts;
        const int4 dn = bn < n_blocks ? blk[bn] : make_int4(0, 0, 0, 0);
        const int nsub = (d.w >> 24) & 7;
        if (!nsub) break;
        {
            const int g = (d.w >> 16) & 7, gn = (d.w >> 20) & 7;
            const int4 wv = *reinterpret_cast<const int4 *>(sw + 4 * g);
            const Wt w[4] = {__builtin_bit_cast(Wt, wv.x), __builtin_bit_cast(Wt, wv.y),
                             __builtin_bit_cast(Wt, wv.z), __builtin_bit_cast(Wt, wv.w)};
            const int r0 = d.y + lane;
            const int r[4] = {r0, r0 + int(short(d.z & 0xffff)), r0 + (d.z >> 16),
                              r0 + int(short(d.w & 0xffff))};
            Acc x[4][4];  // [sub-block][channel]
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nsub) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) x[q][j] = Elem<T>::val(raw[r[j] + 32 * q]);
                }
            Acc v[4];
            if (gn == kSbG) {
                if constexpr (std::is_same<Acc, float>::value) {
#pragma unroll
                    for (int q = 0; q < 4; q += 2) {
                        v[q] = w[0] * x[q][0];
                        v[q + 1] = w[0] * x[q + 1][0];
#pragma unroll
                        for (int j = 1; j < 4; ++j)
                            fma2(v[q], v[q + 1], w[j], w[j], x[q][j], x[q + 1][j]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[q] = w[0] * x[q][0] + w[1] * x[q][1] + w[2] * x[q][2] + w[3] * x[q][3];
                }
            } else {  // the last group of a plan may hold fewer channels
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = w[0] * x[q][0];
#pragma unroll
                    for (int j = 1; j < kSbG; ++j)
                        if (j < gn) v[q] += w[j] * x[q][j];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nsub) P[d.x + 32 * q + lane] = v[q];
        }
        d = dn;
        b = bn;
    }
}

// The packed 16-bit offsets of all the chunk's groups are loaded first, so
// their shared-memory latency is paid once per chunk rather than per group.
template <int DPT>
struct OffWords {
    uint32_t w[DPT / 2];
};
template <int DPT>
__device__ __forceinline__ OffWords<DPT> load_offwords(const uint16_t *p) {
    OffWords<DPT> r;
    if constexpr (DPT == 8) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        r.w[0] = v.x, r.w[1] = v.y, r.w[2] = v.z, r.w[3] = v.w;
    } else if constexpr (DPT == 4) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        r.w[0] = v.x, r.w[1] = v.y;
    } else {
        r.w[0] = *reinterpret_cast<const uint32_t *>(p);
    }
    return r;
}

template <typename Acc, int DPT, int SPT>
__device__ __forceinline__ void sb_trials4(Acc (&acc)[DPT][SPT], const Acc *Pl,
                                           const uint16_t *poffs, int Dt, int ng) {
    OffWords<DPT> ow[4];
#pragma unroll
    for (int g = 0; g < 4; ++g)
        if (g < ng) ow[g] = load_offwords<DPT>(poffs + g * Dt);
#pragma unroll
    for (int g = 0; g < 4; ++g) {  // up to 4 groups (16 channels) at a time
        if (g < ng) {
            int o[DPT];
#pragma unroll
            for (int i = 0; i < DPT / 2; ++i) {
                o[2 * i] = int(ow[g].w[i] & 0xffffu);
                o[2 * i + 1] = int(ow[g].w[i] >> 16);
            }
            // trials of a thread that share the group's series and offset
            // (same pattern, same base delay) reuse the loaded values
            Acc v[SPT];
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                const Acc *src = Pl + o[i];
                if constexpr (std::is_same<Acc, float>::value && SPT % 2 == 0) {
                    if (i == 0 || o[i] != o[i - 1]) {
#pragma unroll
                        for (int j = 0; j < SPT; ++j) v[j] = src[32 * j];
                    }
#pragma unroll
                    for (int j = 0; j < SPT; j += 2)
                        add2(acc[i][j], acc[i][j + 1], v[j], v[j + 1]);
                } else {
#pragma unroll
                    for (int j = 0; j < SPT; ++j) acc[i][j] += src[32 * j];
                }
            }
        }
    }
}

// The trial loop over a chunk's ng groups, four at a time. PASSES: 1 = at
// most 4 groups (16 channels); 2 = up to 8 (32 channels) as two inlined
// passes; 0 = up to 8 as a loop over one copy of the pass. Which form is
// fastest depends on the kernel (GB300, survey scale): the FP32 kinds 2-4
// keep one pass (a second one, even never taken, cost 5.7 %); 8-bit input
// takes two inlined passes (2.26 against 2.32 ms as a loop); 16-bit input
// and kind 6 take the loop (16-bit kind 4: 2.37 against 2.44 ms; FP32 kind
// 6: 2.34 against 2.55 ms, where the inlined form spills).
template <int PASSES, typename Acc, int DPT, int SPT>
__device__ __forceinline__ void sb_trials(Acc (&acc)[DPT][SPT], const Acc *Pl,
                                          const uint16_t *poffs, int Dt, int ng) {
    if constexpr (PASSES == 1) {
        sb_trials4<Acc, DPT, SPT>(acc, Pl, poffs, Dt, ng);
    } else if constexpr (PASSES == 2) {
        sb_trials4<Acc, DPT, SPT>(acc, Pl, poffs, Dt, min(ng, 4));
        if (ng > 4) sb_trials4<Acc, DPT, SPT>(acc, Pl, poffs + 4 * Dt, Dt, ng - 4);
    } else {
#pragma unroll 1
        for (int g0 = 0; g0 < ng; g0 += 4)
            sb_trials4<Acc, DPT, SPT>(acc, Pl, poffs + g0 * Dt, Dt, min(ng - g0, 4));
    }
}

// The trial-loop form of a sub-band kernel (see sb_trials).
template <typename T, bool ONE_SLOT>
__host__ __device__ constexpr int sb_passes() {
    return sizeof(T) == 1 ? 2 : ((ONE_SLOT || sizeof(T) == 2) ? 0 : 1);
}

// kind 2: sub-band partial sums with a producer warp. Warps [0, NC) compute;
// warp NC only stages chunks, running up to `stages` chunks ahead and
// throttled by the slots' empty barriers (one arrival per chunk, made after
// the compute warps' build barrier). Per chunk the compute warps build the
// partial series (and copy the chunk's trial offsets next to them), meet at
// a named barrier, release the staging slot and run the trial loop.
// Partial-sum slots alternate by global chunk parity, so a chunk's build
// never overwrites what slower warps still read. (Replacing the barrier by
// per-warp mbarrier hand-offs, so that a warp builds chunk k+1 before its
// trials on chunk k, measured slower on GB300.)
// ONE_SLOT (kind 6): a single partial-sum slot, so that FP32 input fits
// 32-channel chunks; a second barrier per chunk then keeps the next build
// from overwriting series that slower warps still read.
template <typename T, int DPT, int SPT, bool LIVE, bool ONE_SLOT = false>
__device__ __forceinline__ void fwd_tile_sb(const FwdArgs &a, int dtile, int ttile, int b,
                                            uint64_t *bars, unsigned char *stage0,
                                            uint32_t &kbase) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full = bars, *empty = bars + 8;
    volatile int *gave_up = reinterpret_cast<volatile int *>(&bars[7]);
    const uint32_t S = uint32_t(a.stages);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nc = int(blockDim.x >> 5) - 1;  // compute warps; warp nc produces
    const long long t0 = (long long)ttile * a.Ts;
    const int2 kr = chunk_range<LIVE>(a, dtile, ttile);
    const int n_chunks = kr.y - kr.x;
    const Stager<T> st = make_stager<T>(a, dtile, b, t0, stage0, true, kr.x);
    const uint32_t poffs_bytes = st.tab1_bytes;
    const int pslot_bytes = a.p_elems * int(sizeof(Acc)) + int(poffs_bytes);
    unsigned char *pslot0 = stage0 + S * st.stage_bytes;

    if (warp == nc) {
        // ---------------- producer warp
        // Channel descriptors are loaded kDescAhead chunks before their copy
        // is issued, so the issue rate is not bound by one global-memory
        // latency per chunk.
        // The ring is indexed by compile-time positions (the loop over j is
        // unrolled), so a descriptor is loaded into the register it is
        // consumed from kDescAhead chunks later, with no move that would wait
        // for the load.
        int4 q[kDescAhead];
#pragma unroll
        for (int j = 0; j < kDescAhead; ++j)
            q[j] = j < n_chunks ? st.desc(j, lane) : make_int4(0, 0, 0, 0);
        for (int k0 = 0; k0 < n_chunks; k0 += kDescAhead) {
#pragma unroll
            for (int j = 0; j < kDescAhead; ++j) {
                const int k = k0 + j;
                if (k < n_chunks) {
                    const uint32_t kg = kbase + uint32_t(k);
                    const int slot = int(kg % S);
                    bool ok = true;
                    if (kg >= S)
                        ok = mbar_wait_bounded(&empty[slot], ((kg / S) - 1u) & 1u, a.err,
                                               kWaitBudgetNs, gave_up);
                    if (__all_sync(0xffffffffu, ok)) st.issue(k, slot, q[j], &full[slot], lane);
                    q[j] = k + kDescAhead < n_chunks ? st.desc(k + kDescAhead, lane)
                                                     : make_int4(0, 0, 0, 0);
                }
            }
        }
        kbase += uint32_t(n_chunks);
        return;
    }

    // ---------------- compute warps
    const int wd = warp % a.warps_dm, wt = warp / a.warps_dm;
    Acc acc[DPT][SPT];
#pragma unroll
    for (int i = 0; i < DPT; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = Acc(0);
    const int lb = wt * 32 * SPT + lane;

    for (int k = 0; k < n_chunks; ++k) {
        const uint32_t kg = kbase + uint32_t(k);
        const int slot = int(kg % S);
        // A failed wait sets the give-up flag before the barrier; after it
        // every warp sees the flag and skips the trials on the chunk.
        const bool ok = __all_sync(
            0xffffffffu,
            mbar_wait_bounded(&full[slot], (kg / S) & 1u, a.err, kWaitBudgetNs, gave_up));
        const unsigned char *sb = stage0 + slot * st.stage_bytes;
        const T *raw = reinterpret_cast<const T *>(sb);
        const int4 *bd = reinterpret_cast<const int4 *>(sb + a.stage_data_bytes + poffs_bytes);
        const Wt *sw = reinterpret_cast<const Wt *>(sb + a.stage_data_bytes + st.tab_bytes);
        unsigned char *pb = pslot0 + (ONE_SLOT ? 0u : (kg & 1u)) * pslot_bytes;
        Acc *P = reinterpret_cast<Acc *>(pb);
        uint16_t *poffs = reinterpret_cast<uint16_t *>(pb + a.p_elems * int(sizeof(Acc)));
        const int ng = (min(a.cch, a.C - (kr.x + k) * a.cch) + kSbG - 1) / kSbG;

        if (ok) {
            sb_build_blocks<T>(P, raw, bd, sw, a.n_blocks, warp, nc, lane);
            // the chunk's trial offsets move next to its partial sums
            const uint32_t *src = reinterpret_cast<const uint32_t *>(sb + a.stage_data_bytes);
            uint32_t *dst = reinterpret_cast<uint32_t *>(poffs);
            for (int i = tid; i < int(poffs_bytes / 4); i += nc * 32) dst[i] = src[i];
        }
        compute_barrier(nc * 32);
        if constexpr (ONE_SLOT) {
            // every warp reaches both barriers of a chunk, whatever the flag
            // (the producer may set it between two warps' reads)
            if (!*gave_up) {
                if (tid == 0) mbar_arrive(&empty[slot]);
                sb_trials<sb_passes<T, true>(), Acc, DPT, SPT>(acc, P + lb, poffs + wd * DPT, a.Dt,
                                                               ng);
            }
            compute_barrier(nc * 32);
        } else {
            if (*gave_up) continue;  // no arrival: the producer's next wait fails too
            if (tid == 0) mbar_arrive(&empty[slot]);  // nothing reads this staging slot any more
            sb_trials<sb_passes<T, false>(), Acc, DPT, SPT>(acc, P + lb, poffs + wd * DPT, a.Dt,
                                                            ng);
        }
    }
    kbase += uint32_t(n_chunks);
    if (!*gave_up) store_lane_strided<Acc, DPT, SPT>(a, acc, dtile, b, t0, wd, lb);
}

// kind 3: warp-specialised sub-band. Warps [0, NC) are trial warps (as in
// kind 2), warps [NC, NC + 4) builders. Barriers: full/empty of the staging
// slots at bars[0..3] / bars[8..11], full/empty of the partial-sum slots at
// bars[4..6] / bars[12..14]. A partial-sum slot holds the chunk's partial
// series followed by its per-group trial offsets (copied out of the staging
// slot so that slot can be refilled as soon as the builders are done).
template <typename T, int DPT, int SPT, bool LIVE>
__device__ __forceinline__ void fwd_tile_ws(const FwdArgs &a, int dtile, int ttile, int b,
                                            uint64_t *bars, unsigned char *stage0,
                                            uint32_t &kbase) {
    using Acc = typename Elem<T>::Acc;
    using Wt = typename Elem<T>::W;
    uint64_t *full_r = bars, *empty_r = bars + 8, *full_p = bars + 4, *empty_p = bars + 12;
    volatile int *gave_up = reinterpret_cast<volatile int *>(&bars[7]);
    const uint32_t S = uint32_t(a.stages), Q = uint32_t(kWsPSlots);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nc = int(blockDim.x >> 5) - kWsBuilders;  // trial warps
    const long long t0 = (long long)ttile * a.Ts;
    const int2 kr = chunk_range<LIVE>(a, dtile, ttile);
    const int n_chunks = kr.y - kr.x;
    const Stager<T> st = make_stager<T>(a, dtile, b, t0, stage0, true, kr.x);
    const uint32_t poffs_bytes = st.tab1_bytes;
    const int pslot_bytes = a.p_elems * int(sizeof(Acc)) + int(poffs_bytes);
    unsigned char *pslot0 = stage0 + S * st.stage_bytes;

    if (warp >= nc) {
        // ---------------- builder warps
        const int bw = warp - nc;
        auto issue = [&](int k, int4 dsc) {  // builder warp 0
            const uint32_t kg = kbase + uint32_t(k);
            const int slot = int(kg % S);
            bool ok = true;
            if (kg >= S)
                ok = mbar_wait_bounded(&empty_r[slot], ((kg / S) - 1u) & 1u, a.err, kWaitBudgetNs,
                                       gave_up);
            if (__all_sync(0xffffffffu, ok && !*gave_up))
                st.issue(k, slot, dsc, &full_r[slot], lane);
        };
        if (bw == 0) {
            const int pro = min(int(S), n_chunks);
            for (int k = 0; k < pro; ++k) issue(k, st.desc(k, lane));
        }
        for (int k = 0; k < n_chunks; ++k) {
            const uint32_t kg = kbase + uint32_t(k);
            const int rs = int(kg % S), ps = int(kg % Q);
            const int kn = k - 1 + int(S);
            int4 pre = make_int4(0, 0, 0, 0);
            if (bw == 0 && k >= 1 && kn < n_chunks) pre = st.desc(kn, lane);
            bool ok = mbar_wait_bounded(&full_r[rs], (kg / S) & 1u, a.err, kWaitBudgetNs, gave_up);
            if (ok && kg >= Q)
                ok = mbar_wait_bounded(&empty_p[ps], ((kg / Q) - 1u) & 1u, a.err, kWaitBudgetNs,
                                       gave_up);
            if (!__all_sync(0xffffffffu, ok)) break;  // a lost hand-off ends the tile
            const unsigned char *sb = stage0 + rs * st.stage_bytes;
            const T *raw = reinterpret_cast<const T *>(sb);
            const int4 *bd =
                reinterpret_cast<const int4 *>(sb + a.stage_data_bytes + poffs_bytes);
            const Wt *sw = reinterpret_cast<const Wt *>(sb + a.stage_data_bytes + st.tab_bytes);
            unsigned char *pb = pslot0 + ps * pslot_bytes;
            sb_build_blocks<T>(reinterpret_cast<Acc *>(pb), raw, bd, sw, a.n_blocks, bw,
                               kWsBuilders, lane);
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
            if (bw == 0 && k >= 1 && kn < n_chunks) issue(kn, pre);
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
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full_p[ps], (kg / Q) & 1u, a.err,
                                                       kWaitBudgetNs, gave_up)))
            break;
        const unsigned char *pb = pslot0 + ps * pslot_bytes;
        const uint16_t *poffs =
            reinterpret_cast<const uint16_t *>(pb + a.p_elems * int(sizeof(Acc))) + wd * DPT;
        const int ng = (min(a.cch, a.C - (kr.x + k) * a.cch) + kSbG - 1) / kSbG;
        sb_trials<sb_passes<T, false>(), Acc, DPT, SPT>(
            acc, reinterpret_cast<const Acc *>(pb) + lb, poffs, a.Dt, ng);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_p[ps]);
    }
    kbase += uint32_t(n_chunks);
    if (!*gave_up) store_lane_strided<Acc, DPT, SPT>(a, acc, dtile, b, t0, wd, lb);
}

// Dispatches a tile to the kind's body.
template <int KIND, typename T, int DPT, int SPT, bool LIVE = false>
__device__ __forceinline__ void fwd_tile_any(const FwdArgs &a, int dtile, int ttile, int b,
                                             uint64_t *bars, unsigned char *stage0,
                                             uint32_t &kbase) {
    if constexpr (KIND == 2 || KIND == 4)
        fwd_tile_sb<T, DPT, SPT, LIVE>(a, dtile, ttile, b, bars, stage0, kbase);
    else if constexpr (KIND == 6)
        fwd_tile_sb<T, DPT, SPT, LIVE, true>(a, dtile, ttile, b, bars, stage0, kbase);
    else if constexpr (KIND == 3)
        fwd_tile_ws<T, DPT, SPT, LIVE>(a, dtile, ttile, b, bars, stage0, kbase);
    else
        fwd_tile<KIND, T, DPT, SPT, LIVE>(a, dtile, ttile, b, bars, stage0, kbase);
}

}  // namespace dd
