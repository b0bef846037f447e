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
#include <algorithm>

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
constexpr int64_t kMaxRecords = (int64_t)kMaxBlocks * kThreadsPerBlock * kRecordsPerThread;   // 1,048,576
constexpr size_t kTicketBytes = 256;
constexpr size_t kScratchBytes = kTicketBytes + (size_t)kMaxBlocks * kStatVals * sizeof(double);  // 131,328

// ticket (first 4 bytes of a 256-byte slot), then kMaxBlocks x 8 partials
static __device__ __align__(256) unsigned char g_wall_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];      // device address of g_wall_scratch, per device

}  // namespace

extern "C" int wmibm_wall_stress_noalloc(wmibm_handle *h, const void *u, const void *v, const void *w,
                                         void *const tau[6], wmibm_band_stats *stats, void *stream_)
{
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

    // set-up, once per device, with that device current: the host-side name of
    // a __device__ array is not a device address
    if (g_scratch_addr[h->device] == nullptr) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_wall_scratch);
        if (e != cudaSuccess) return cuda_status(h, e, "cudaGetSymbolAddress(g_wall_scratch)");
        g_scratch_addr[h->device] = ptr;
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[h->device];
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
