// Host-side state shared by the launchers: the per-thread launch counter and
// the per-device SM counts.
#include "sfe_internal.cuh"

namespace sfe {

thread_local unsigned long long g_launches = 0;

int device_sms() {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (dev < 0 || dev >= kMaxDevices) dev = kMaxDevices - 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    if (n <= 0) return 1;
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

}  // namespace sfe
