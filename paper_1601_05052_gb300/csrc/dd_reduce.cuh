// dd_reduce.cuh -- deterministic FP32 sums for the weight-gradient
// reductions.
//
// fixed_order_sum adds n values p[0], p[stride], ... in FP32 in an order
// that depends on n alone: runs of 8 consecutive values are summed in turn,
// and the run sums are combined pairwise as a binary counter combines its
// carries (the pairwise summation of a balanced tree over the runs). The
// error grows with log2(n / 8) rather than n, and the same inputs give the
// same bits on every call.
#pragma once

namespace dd {

__device__ __forceinline__ float fixed_order_sum(const float *p, long long n, long long stride) {
    constexpr int kRun = 8;
    float part[40];  // pending sums of 2^k runs; 40 levels exceed any n here
    int level[40];
    int top = 0;
    for (long long i = 0; i < n; i += kRun) {
        float s = 0.f;
        const long long e = i + kRun < n ? i + kRun : n;
        for (long long j = i; j < e; ++j) s += p[j * stride];
        int lv = 0;
        while (top > 0 && level[top - 1] == lv) {  // equal-sized neighbours merge
            s = part[top - 1] + s;
            --top;
            ++lv;
        }
        part[top] = s;
        level[top] = lv;
        ++top;
    }
    float s = 0.f;
    while (top > 0) s = part[--top] + s;  // smallest pending sums first
    return s;
}

}  // namespace dd
