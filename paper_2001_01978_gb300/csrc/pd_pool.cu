// pd_pool.cu -- process-wide cache of the library's device allocations.
//
// A solver handle needs a Lanczos window and work vectors whose sizes depend
// only on (Omega, N, window).  A caller that creates and destroys handles in a
// loop (a mean-field iteration solves the same sizes again and again) would
// otherwise pay cudaMalloc and cudaFree for every handle.  Freed blocks are
// kept per device, keyed by their rounded size, and handed out again; when
// cudaMalloc runs out of memory the cache is emptied once and the allocation
// retried.  pairdiag_release_cache() returns every cached block to the driver.
#include "pd_internal.h"
#include "pairdiag.h"

#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

namespace pd {
namespace {

struct Pool {
    std::mutex mu;
    std::unordered_map<void *, std::pair<int, size_t>> live;       // block -> (device, rounded size)
    std::map<std::pair<int, size_t>, std::vector<void *>> cached;  // (device, rounded size) -> free blocks
};

Pool &pool()
{
    static Pool *p = new Pool;   // never destroyed: blocks may be freed during static destruction
    return *p;
}

// 512 bytes up to 1 MiB, then whole 2 MiB pages, so that a block serves
// requests that differ by less than its granularity
size_t round_size(size_t bytes)
{
    if (bytes == 0) bytes = 16;
    const size_t g = bytes <= (size_t(1) << 20) ? 512 : (size_t(2) << 20);
    return (bytes + g - 1) / g * g;
}

// cudaFree every cached block (caller holds the lock)
void release_locked(Pool &P)
{
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : P.cached) {
        if (kv.second.empty()) continue;
        cudaSetDevice(kv.first.first);
        for (void *q : kv.second) cudaFree(q);
        kv.second.clear();
    }
    cudaSetDevice(cur);
}

}  // namespace

cudaError_t pool_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t sz = round_size(bytes);
    Pool &P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.cached.find({dev, sz});
    if (it != P.cached.end() && !it->second.empty()) {
        *p = it->second.back();
        it->second.pop_back();
        P.live[*p] = {dev, sz};
        return cudaSuccess;
    }
    e = cudaMalloc(p, sz);
    if (e == cudaErrorMemoryAllocation) {       // give the cached blocks back and retry once
        cudaGetLastError();
        release_locked(P);
        e = cudaMalloc(p, sz);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    P.live[*p] = {dev, sz};
    return cudaSuccess;
}

void pool_free(void *p)
{
    if (!p) return;
    Pool &P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.live.find(p);
    if (it == P.live.end()) {                    // not from the pool
        cudaFree(p);
        return;
    }
    P.cached[it->second].push_back(p);
    P.live.erase(it);
}

size_t pool_cached_bytes()
{
    Pool &P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    size_t total = 0;
    for (auto &kv : P.cached) total += kv.first.second * kv.second.size();
    return total;
}

}  // namespace pd

extern "C" int pairdiag_release_cache(size_t *released_bytes)
{
    pd::Pool &P = pd::pool();
    std::lock_guard<std::mutex> lock(P.mu);
    size_t total = 0;
    for (auto &kv : P.cached) total += kv.first.second * kv.second.size();
    pd::release_locked(P);
    if (released_bytes) *released_bytes = total;
    return PD_OK;
}
