// Wall model at the band nodes (Sec. 3.3 of Liu & Stevens, arXiv:2006.03343),
// stand-alone form.
//
// One thread per band node evaluates the model of band.cuh from the node's
// precomputed record (trilinear stencils of u, v on the uv-grid and w on the
// w-grid at x_c, unit normal, log-law factor) and writes its stress
// components; extra blocks of the same launch zero the solid-node stresses.
// Band statistics are reduced per warp with shuffles, per block in shared
// memory, and across blocks by the last block to finish (fixed order, so the
// result is deterministic).
#include "band.cuh"

using namespace wmibm;

namespace {

template <typename T>
struct WSParams {
    const void *u, *v, *w;
    T *txx, *txy, *tyy, *tzz, *txz, *tyz;
    const void *rec;
    const int32_t *solid_w, *solid_uv;
    int64_t nb_w, nb_uv, ns_w, ns_uv;
    int32_t nx, ny;
    int64_t plane;
    unsigned band_blocks;
    T *partials;
    unsigned int *ticket;
    wmibm_band_stats *stats;
    const T *logz0;          // optional per-cell log z0 (C then computed per call)
    T log_phi_c, kappa2;
};

template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) k_wall_stress(WSParams<T> p)
{
    __shared__ T red[32][kStatVals];

    if (blockIdx.x >= p.band_blocks) {
        // solid nodes: the stress is set to zero (Sec. 3.3)
        const int64_t t = (int64_t)(blockIdx.x - p.band_blocks) * kThreads + threadIdx.x;
        if (t < p.ns_w) {
            const int32_t idx = __ldg(p.solid_w + t);
            p.txz[idx] = T(0);
            p.tyz[idx] = T(0);
        } else if (t < p.ns_w + p.ns_uv) {
            const int32_t idx = __ldg(p.solid_uv + (t - p.ns_w));
            p.txx[idx] = T(0);
            p.txy[idx] = T(0);
            p.tyy[idx] = T(0);
            p.tzz[idx] = T(0);
        }
        return;
    }

    T acc[kStatVals];
    stats_identity(acc);
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t < p.nb_w + p.nb_uv) {
        const bool is_w = t < p.nb_w;
        const BandOut<T> o = band_model<T, V>(p.rec, t, is_w, reinterpret_cast<const V *>(p.u),
                                              reinterpret_cast<const V *>(p.v), reinterpret_cast<const V *>(p.w),
                                              p.nx, p.ny, p.plane, p.logz0, p.log_phi_c, p.kappa2);
        if (is_w) {
            p.txz[o.idx] = o.t0;
            p.tyz[o.idx] = o.t1;
        } else {
            p.txx[o.idx] = o.t0;
            p.txy[o.idx] = o.t1;
            p.tyy[o.idx] = o.t2;
            p.tzz[o.idx] = o.t3;
        }
        stats_add(acc, is_w ? 0 : 1, o.tw, o.ur);
    }

    if (p.stats == nullptr) return;            // uniform across the launch
    stats_block_reduce(acc, red);
    stats_finish(acc, red, p.partials, p.ticket, p.band_blocks, p.stats, p.nb_w, p.nb_uv);
}

template <typename T, typename V>
int launch(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
           wmibm_band_stats *stats, cudaStream_t stream, const T *logz0)
{
    WSParams<T> p;
    p.u = u; p.v = v; p.w = w;
    p.txx = (T *)tau[0]; p.txy = (T *)tau[1]; p.tyy = (T *)tau[2];
    p.tzz = (T *)tau[3]; p.txz = (T *)tau[4]; p.tyz = (T *)tau[5];
    p.rec = h->rec;
    p.solid_w = h->lists.p[WMIBM_LIST_SOLID_W];
    p.solid_uv = h->lists.p[WMIBM_LIST_SOLID_UV];
    p.nb_w = h->lists.n[WMIBM_LIST_BAND_W];
    p.nb_uv = h->lists.n[WMIBM_LIST_BAND_UV];
    p.ns_w = h->lists.n[WMIBM_LIST_SOLID_W];
    p.ns_uv = h->lists.n[WMIBM_LIST_SOLID_UV];
    p.nx = h->nx; p.ny = h->ny;
    p.plane = (int64_t)h->nx * h->ny;
    p.band_blocks = (unsigned)((p.nb_w + p.nb_uv + kThreads - 1) / kThreads);
    p.partials = (T *)h->partials;
    p.ticket = h->ticket;
    p.stats = stats;
    p.logz0 = logz0;
    p.log_phi_c = (T)log(h->phi_c);
    p.kappa2 = (T)(h->kappa * h->kappa);
    const unsigned solid_blocks = (unsigned)((p.ns_w + p.ns_uv + kThreads - 1) / kThreads);
    if (stats && p.band_blocks == 0) {
        cudaError_t e = cudaMemsetAsync(stats, 0, 2 * sizeof(wmibm_band_stats), stream);
        if (e != cudaSuccess) return cuda_status(h, e, "clear stats");
    }
    if (p.band_blocks + solid_blocks == 0) return WMIBM_OK;
    k_wall_stress<T, V><<<p.band_blocks + solid_blocks, kThreads, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_wall_stress launch");
}

}  // namespace

namespace wmibm {

int wall_stress_impl(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                     wmibm_band_stats *stats, cudaStream_t stream, const void *logz0)
{
    if (h->dtype == WMIBM_F64) return launch<double, double>(h, u, v, w, tau, stats, stream, (const double *)logz0);
    if (h->vel_dtype == WMIBM_BF16)
        return launch<float, __nv_bfloat16>(h, u, v, w, tau, stats, stream, (const float *)logz0);
    return launch<float, float>(h, u, v, w, tau, stats, stream, (const float *)logz0);
}

}  // namespace wmibm

extern "C" int wmibm_wall_stress(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                                 wmibm_band_stats *stats, void *stream)
{
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w || !tau) return set_error(h, WMIBM_EINVAL, "NULL velocity or stress pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    int st = check_device(h);
    if (st) return st;
    return wall_stress_impl(h, u, v, w, tau, stats, (cudaStream_t)stream, nullptr);
}
