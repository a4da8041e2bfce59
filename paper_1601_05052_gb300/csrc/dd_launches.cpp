// dd_launches.cpp -- LaunchTracker: the events a plan, batch or adjoint state
// records on the streams its kernels were launched on, so that replacing its
// device tables (or arguments) waits for its own earlier launches only.
#include "dd_internal.h"

namespace dd {

void LaunchTracker::note(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: treat as captured (keeps tables)
    }
    std::lock_guard<std::mutex> lk(mu);
    if (cs != cudaStreamCaptureStatusNone) {
        captured = true;
        return;
    }
    ++clock;
    int i = 0;
    while (i < n && stream[i] != s) ++i;
    if (i == n && n == kMax) {
        // every slot is taken: the least recently used stream's last launch
        // is waited for here, after which that slot can forget it
        i = 0;
        for (int j = 1; j < n; ++j)
            if (used[j] < used[i]) i = j;
        if (cudaEventSynchronize(event[i]) != cudaSuccess) {
            cudaGetLastError();
            overflow = true;
        }
        stream[i] = s;
    } else if (i == n) {
        if (cudaEventCreateWithFlags(&event[n], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            overflow = true;
            return;
        }
        stream[n++] = s;
    }
    used[i] = clock;
    if (cudaEventRecord(event[i], s) != cudaSuccess) {
        cudaGetLastError();
        overflow = true;
    }
}

cudaError_t LaunchTracker::wait() {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaEventSynchronize(event[i]);
        if (e != cudaSuccess) return e;
    }
    if (overflow) return cudaDeviceSynchronize();
    return cudaSuccess;
}

cudaError_t LaunchTracker::order_before(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(mu);
    if (overflow) return cudaDeviceSynchronize();
    for (int i = 0; i < n; ++i) {
        if (stream[i] == s) continue;  // stream order covers it
        cudaError_t e = cudaStreamWaitEvent(s, event[i], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void LaunchTracker::destroy() {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; ++i) cudaEventDestroy(event[i]);
    n = 0;
}

}  // namespace dd
