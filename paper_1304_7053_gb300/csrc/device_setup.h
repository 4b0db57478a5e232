// Per-device launch set-up shared by every launcher.
//
// Function attributes (the dynamic shared-memory limit) and occupancy apply
// to the device that is current when they are set or queried, so each is
// kept per device: a process that drives several GPUs sets the attribute on
// each of them before its first launch there.  The "attribute set" flags are
// atomic bit masks (one bit per device), safe to test and set from several
// host threads; the occupancy caches are per thread and per device.
#pragma once

#include <atomic>
#include <cstddef>

#include <cuda_runtime.h>

namespace sbg {

constexpr int kMaxDevices = 64;

// The current device, or -1 when it cannot be queried or is out of range.
inline int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

// One bit per device: the set-up step has been done there.
struct DeviceFlags {
    std::atomic<unsigned long long> bits{0};
    bool test(int dev) const { return (bits.load(std::memory_order_acquire) >> dev) & 1ull; }
    void set(int dev) { bits.fetch_or(1ull << dev, std::memory_order_acq_rel); }
};

// Raise the kernel's dynamic shared-memory limit on the current device once.
// Two threads may both make the (idempotent) call the first time.
template <class Kern>
inline cudaError_t ensure_smem_limit(Kern kern, int bytes, DeviceFlags& done) {
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    if (done.test(dev)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.set(dev);
    return e;
}

// Resident blocks per SM of one kernel for one dynamic shared-memory size,
// cached per device (the query costs microseconds of host time per call).
struct OccCache {
    size_t smem[kMaxDevices];
    int val[kMaxDevices];
    OccCache() {
        for (int d = 0; d < kMaxDevices; ++d) { smem[d] = ~(size_t)0; val[d] = 0; }
    }
};

template <class Kern>
inline cudaError_t blocks_per_sm(Kern kern, int threads, size_t smem, OccCache& cache, int* out) {
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    if (cache.smem[dev] == smem) { *out = cache.val[dev]; return cudaSuccess; }
    int v = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem);
    if (e != cudaSuccess) return e;
    cache.smem[dev] = smem;
    cache.val[dev] = v;
    *out = v;
    return cudaSuccess;
}

}  // namespace sbg
