// Device memory of libfdtd: a library-owned stream-ordered pool per device, host-side injection of
// allocation failures, and the timeout-injection diagnostic.
#include "api_internal.h"

namespace fdtd {

// Device memory comes from a library-owned stream-ordered pool per device that keeps freed
// memory for reuse (release threshold: never), so creating and destroying contexts at a
// serving rate neither returns memory to the driver nor synchronises the device.
cudaMemPool_t lib_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = pool;
    return pool;
}

// Host-side fault injection (fdtd_debug_fail_alloc): the allocation that counts this down to zero fails.
std::atomic<int> g_fail_alloc_in{-1};

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    for (int n = g_fail_alloc_in.load(); n >= 0;)
        if (g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {
            if (n == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    cudaMemPool_t pool = lib_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaError_t dmalloc(fdtd_ctx *c, void **p, size_t bytes) {
    cudaError_t e = pool_alloc(p, bytes, c->stream);
    if (e == cudaSuccess) c->bytes += (long long)bytes;
    return e;
}

}  // namespace fdtd

using namespace fdtd;

extern "C" {

int fdtd_debug_fail_alloc(int after) {
    g_fail_alloc_in.store(after < 0 ? -1 : after);
    return FDTD_OK;
}

int fdtd_debug_inject_timeout(fdtd_ctx *c, int limit_us) {
    if (!c) return FDTD_ERR_ARG;
    if (limit_us < 1 || limit_us > 1000000) return fail(c, FDTD_ERR_ARG, "limit_us must be in [1, 1e6]");
    if (!use_fused(c)) return fail(c, FDTD_ERR_STATE, "timeout injection needs the fused kernel");
    c->inject_us = limit_us;
    return FDTD_OK;
}

}  // extern "C"
