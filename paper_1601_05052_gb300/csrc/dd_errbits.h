// dd_errbits.h -- bits of a plan's device error word, written by kernels and
// read back by dd_plan_check_device().
#pragma once

namespace dd {
constexpr int kErrWaitTimeout = 1;  // an mbarrier wait ran out of its time budget
constexpr int kErrBadIndex = 2;     // a bounds check failed
}  // namespace dd
