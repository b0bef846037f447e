// wmibm_wall_stress_noalloc: the wall-model call with its reduction scratch in
// a static device array instead of memory the handle allocated.
//
// Some callers cannot allocate device memory at the time they call: code that
// runs while a CUDA graph is being captured (cudaMalloc is not a legal stream
// operation there), plug-ins hosted by a framework that owns the device memory
// pool, or real-time loops that must not touch the allocator.  This entry point
// allocates nothing: the per-block partial statistics and the last-block ticket
// of the wall kernel live in g_wall_scratch below, which every GPU that loads
// the library holds until the process exits.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "internal.cuh"

using namespace wmibm;

namespace wmibm {
int wall_model_with_scratch(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                            wmibm_band_stats *stats, void *partials, unsigned *ticket, unsigned blocks,
                            cudaStream_t stream);
}

namespace {

constexpr int kThreadsPerBlock = 256;
constexpr int kRecordsPerThread = 2;
constexpr unsigned kMaxBlocks = 2048;                                   // blocks of the wall kernel
// The array bounds only the number of blocks (one partial per block); the kernel
// walks any number of records with a grid stride.  The record limit is a choice:
// one call stays within one pass of its grid, two records per thread.
constexpr int64_t kMaxRecords = (int64_t)kMaxBlocks * kThreadsPerBlock * kRecordsPerThread;   // 1,048,576
constexpr size_t kTicketBytes = 256;
constexpr size_t kScratchBytes = kTicketBytes + (size_t)kMaxBlocks * kStatVals * sizeof(double);  // 131,328

// ticket (first 4 bytes of a 256-byte slot), then kMaxBlocks x 8 partials
static __device__ __align__(256) unsigned char g_wall_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// Device address of g_wall_scratch per device, with the id of the context it was
// looked up in: the module, and with it the array, moves when a device's context
// is made again (after cudaDeviceReset, for instance), so a new context means a
// new look-up.  Filled under a lock; several host threads may call at once.
struct ScratchSlot {
    unsigned long long ctx_id;
    void *addr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_lock;

// Id of the calling thread's current context (driver entry points found once at
// run time, so that the library needs no link to the driver library); 0 where the
// driver offers none.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
std::once_flag g_entry_once;
std::atomic<CtxGetCurrentFn> g_ctx_get_current{nullptr};
std::atomic<CtxGetIdFn> g_ctx_get_id{nullptr};

unsigned long long current_context_id()
{
    std::call_once(g_entry_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current.store(reinterpret_cast<CtxGetCurrentFn>(f));
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id.store(reinterpret_cast<CtxGetIdFn>(f));
    });
    CtxGetCurrentFn get_current = g_ctx_get_current.load();
    CtxGetIdFn get_id = g_ctx_get_id.load();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

}  // namespace

extern "C" int wmibm_wall_stress_noalloc(wmibm_handle *h, const void *u, const void *v, const void *w,
                                         void *const tau[6], wmibm_band_stats *stats, void *stream_)
{
    ApiRange nvtx_range("wmibm_wall_stress_noalloc");
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w || !tau) return set_error(h, WMIBM_EINVAL, "NULL velocity or stress pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    int st = check_device(h);
    if (st) return st;
    if (h->nrec > kMaxRecords)
        return set_error(h, WMIBM_EINVAL,
                         "the band has %lld nodes; wmibm_wall_stress_noalloc handles at most %lld (static scratch "
                         "of %u blocks); use wmibm_wall_stress",
                         (long long)h->nrec, (long long)kMaxRecords, kMaxBlocks);
    if (h->device < 0 || h->device >= kMaxDevices)
        return set_error(h, WMIBM_EINVAL, "device %d beyond the %d devices this entry point serves", h->device,
                         kMaxDevices);

    // set-up, once per device (and again when its context was made anew), with that
    // device current: the host-side name of a __device__ array is not a device address
    unsigned char *base = nullptr;
    {
        const unsigned long long ctx = current_context_id();
        std::lock_guard<std::mutex> lock(g_scratch_lock);
        ScratchSlot &slot = g_scratch[h->device];
        if (slot.addr == nullptr || slot.ctx_id != ctx) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_wall_scratch);
            if (e != cudaSuccess) return cuda_status(h, e, "cudaGetSymbolAddress(g_wall_scratch)");
            slot.addr = ptr;
            slot.ctx_id = ctx;
        }
        base = (unsigned char *)slot.addr;
    }
    unsigned *ticket = (unsigned *)base;
    void *partials = base + kTicketBytes;

    if (stats && h->nrec == 0) {
        cudaError_t e = cudaMemsetAsync(stats, 0, 2 * sizeof(wmibm_band_stats), stream);
        if (e != cudaSuccess) return cuda_status(h, e, "clear stats");
        stats = nullptr;
    }
    // the array keeps the last call's contents: the ticket must start at zero
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return cuda_status(h, e, "clear ticket");

    const int64_t need = (h->nrec + (int64_t)kThreadsPerBlock * kRecordsPerThread - 1) /
                         ((int64_t)kThreadsPerBlock * kRecordsPerThread);
    int64_t blocks = std::max<int64_t>(need, 4 * (int64_t)h->sm_count);
    if (blocks > (int64_t)kMaxBlocks) blocks = kMaxBlocks;
    if (blocks < 1) blocks = 1;
    return wall_model_with_scratch(h, u, v, w, tau, stats, partials, ticket, (unsigned)blocks, stream);
}
