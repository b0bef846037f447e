// C ABI entry of the wall model at the band nodes (Sec. 3.3 of Liu & Stevens,
// arXiv:2006.03343).  The work is done by the persistent wall kernel of
// stencil.cu: every thread of the grid evaluates band records (trilinear
// stencils of u, v on the uv-grid and w on the w-grid at x_c, tangential part,
// log law, rotated stress) and warps zero the solid runs; band statistics are
// reduced per warp and per block into an FP64 accumulator, which a one-thread
// launch converts into the caller's stats.
#include "internal.cuh"

using namespace wmibm;

namespace wmibm {
int wall_model(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
               wmibm_band_stats *stats, const void *logz0, cudaStream_t stream, bool emit);

int wall_stress_impl(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                     wmibm_band_stats *stats, cudaStream_t stream, const void *logz0)
{
    return wall_model(h, u, v, w, tau, stats, logz0, stream, true);
}
}  // namespace wmibm

extern "C" int wmibm_wall_stress(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                                 wmibm_band_stats *stats, void *stream)
{
    ApiRange nvtx_range("wmibm_wall_stress");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w || !tau) return set_error(h, WMIBM_EINVAL, "NULL velocity or stress pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    int st = check_device(h);
    if (st) return st;
    return wall_stress_impl(h, u, v, w, tau, stats, (cudaStream_t)stream, h->logz0);
}
