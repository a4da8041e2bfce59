// dd_kinds.h -- the forward kernel kinds and their CTA shapes, shared by the
// host code that builds a variant's tables and the kernels that run it.
//
// kind 0: lane-strided accumulation from the staged channel windows;
// kind 1: register windows; kind 2: sub-band partial series (groups of four
// channels) with a producer warp; kind 3: kind 2 with warp-specialised
// builders; kind 4: kind 2 in CTAs of up to 16 trial warps; kind 5: kind 0
// with operand reuse between trials that share a channel's delay; kind 6:
// kind 4 with one partial-sum slot and up to 8 groups per chunk, which lets
// FP32 input stage 32 channels at a time.
#pragma once

#include <cuda_runtime.h>

namespace dd {

// Builder warps of kind 3.
constexpr int kWsBuilders = 4;

// Warps a CTA has beyond its warps_dm * warps_time trial warps.
__host__ __device__ constexpr int extra_warps(int kind) {
    return kind == 3 ? kWsBuilders : ((kind == 2 || kind == 4 || kind == 6) ? 1 : 0);
}
// Sub-band kinds (partial series per channel group).
__host__ __device__ constexpr bool is_subband(int kind) {
    return kind == 2 || kind == 3 || kind == 4 || kind == 6;
}
// Largest trial-warp count of a CTA.
__host__ __device__ constexpr int max_trial_warps(int kind) {
    return (kind == 4 || kind == 6) ? 16 : 8;
}
// Launch bounds of the forward kernels: threads per CTA and resident CTAs
// per SM that the register allocation must allow.
__host__ __device__ constexpr int fwd_max_threads(int kind) {
    return 32 * (max_trial_warps(kind) + extra_warps(kind));
}
__host__ __device__ constexpr int fwd_min_blocks(int kind, int dpt, int spt) {
    return kind == 2 ? (dpt * spt <= 16 ? 3 : 2) : (kind == 3 ? 2 : 1);
}

}  // namespace dd
