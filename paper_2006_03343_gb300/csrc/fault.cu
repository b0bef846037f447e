// Failure injection, for testing the error paths of the library.
//  - WMIBM_FAULT=alloc:N when wmibm_init or wmibm_batch_create starts: the N-th
//    allocation the library makes from then on (device or host, counted in the
//    order they are made) fails as if the memory were exhausted; every other
//    allocation goes through.
//  - WMIBM_FAULT=hold_release when a handle or batch is made: its single-launch
//    forms never count their blocks as done with the wall model, so the bounded
//    waits of their dirty stages run out (ETIMEOUT from wmibm_device_status)
//    instead of completing; nothing waits without a limit.
//  - WMIBM_WAIT_LIMIT_NS: the limit of every bounded wait of that handle or batch
//    (default one second).
// Unset, these inject nothing.
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.cuh"

namespace {
std::atomic<long long> g_fail_at{0};     // 1-based number of the allocation to fail; 0: none
std::atomic<long long> g_count{0};       // allocations counted since the last arm
}  // namespace

namespace wmibm {

void fault_arm()
{
    const char *e = getenv("WMIBM_FAULT");
    long long n = 0;
    if (e && strncmp(e, "alloc:", 6) == 0) n = atoll(e + 6);
    g_count.store(0);
    g_fail_at.store(n > 0 ? n : 0);
}

bool fault_fires()
{
    const long long at = g_fail_at.load();
    if (at <= 0) return false;
    return g_count.fetch_add(1) + 1 == at;
}

void fault_wait_settings(uint64_t *wait_ns, int *hold_release)
{
    const char *w = getenv("WMIBM_WAIT_LIMIT_NS");
    double ns = w ? atof(w) : 1e9;
    if (!(ns >= 1e5)) ns = ns > 0 ? 1e5 : 1e9;
    if (ns > 1e10) ns = 1e10;
    *wait_ns = (uint64_t)ns;
    const char *e = getenv("WMIBM_FAULT");
    *hold_release = (e && strcmp(e, "hold_release") == 0) ? 1 : 0;
}

cudaError_t dev_alloc_bytes(void **p, size_t bytes)
{
    if (fault_fires()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void *host_alloc(size_t bytes)
{
    if (fault_fires()) return nullptr;
    return calloc(1, bytes);
}

}  // namespace wmibm
