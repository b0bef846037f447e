// Immersed-boundary velocity condition (Sec. 3.2, Eq. 27 of Liu & Stevens,
// arXiv:2006.03343): u*_IB = u* where phi > 0 and 3 dt/2 grad p^{t-dt} where
// phi <= 0; with no pressure gradient given the body velocity is set to zero.
// Driven by the ascending body-node lists built at init, so only the body
// nodes are touched.  Also the one-pass step entry point.
#include "internal.cuh"

using namespace wmibm;

namespace {

template <typename T, typename V>
struct MaskParams {
    V *u, *v, *w;
    const T *gpx, *gpy, *gpz;
    const int32_t *body_w, *body_uv;
    int64_t nb_w, nb_uv;
    T c;   // 3 dt / 2
};

template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) k_mask(MaskParams<T, V> p)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t < p.nb_uv) {
        const int32_t idx = __ldg(p.body_uv + t);
        const T a = p.gpx ? p.c * __ldg(p.gpx + idx) : T(0);
        const T b = p.gpy ? p.c * __ldg(p.gpy + idx) : T(0);
        p.u[idx] = to_vel<V, T>(a);
        p.v[idx] = to_vel<V, T>(b);
    } else if (t < p.nb_uv + p.nb_w) {
        const int32_t idx = __ldg(p.body_w + (t - p.nb_uv));
        const T a = p.gpz ? p.c * __ldg(p.gpz + idx) : T(0);
        p.w[idx] = to_vel<V, T>(a);
    }
}

template <typename T, typename V>
int launch(wmibm_handle *h, void *u, void *v, void *w, const void *const gradp[3], double dt, cudaStream_t stream)
{
    MaskParams<T, V> p;
    p.u = (V *)u; p.v = (V *)v; p.w = (V *)w;
    p.gpx = gradp ? (const T *)gradp[0] : nullptr;
    p.gpy = gradp ? (const T *)gradp[1] : nullptr;
    p.gpz = gradp ? (const T *)gradp[2] : nullptr;
    p.body_w = h->lists.p[WMIBM_LIST_BODY_W];
    p.body_uv = h->lists.p[WMIBM_LIST_BODY_UV];
    p.nb_w = h->lists.n[WMIBM_LIST_BODY_W];
    p.nb_uv = h->lists.n[WMIBM_LIST_BODY_UV];
    p.c = (T)(1.5 * dt);
    const int64_t total = p.nb_w + p.nb_uv;
    if (total == 0) return WMIBM_OK;
    k_mask<T, V><<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_mask launch");
}

}  // namespace

namespace wmibm {
int wall_stress_impl(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                     wmibm_band_stats *stats, cudaStream_t stream, const void *logz0);
int force_impl(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream, int bx,
               int by, int kc);
void force_default_tile(const wmibm_handle *h, int *bx, int *by, int *kc);
int force_any(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream);
bool stencil_config(const wmibm_handle *h, const void *const tau[6], void *const f[3], StencilConfig *out);
int stencil_force_mask(wmibm_handle *h, void *u, void *v, void *w, const void *const tau[6], void *const f[3],
                       const void *const gradp[3], double dt, const StencilConfig &c, bool pdl, cudaStream_t stream,
                       wmibm_band_stats *emit);
int stencil_force(wmibm_handle *h, const void *const tau[6], void *const f[3], const StencilConfig &c,
                  cudaStream_t stream, wmibm_band_stats *emit);
int wall_model(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
               wmibm_band_stats *stats, const void *logz0, cudaStream_t stream, bool emit);
int mask_impl(wmibm_handle *h, void *u, void *v, void *w, const void *const gradp[3], double dt, cudaStream_t stream);
int stencil_step_fused(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *const f[3],
                       const void *const gradp[3], double dt, int do_mask, wmibm_band_stats *stats,
                       const StencilConfig &c, cudaStream_t stream);

// Wall stress + force (+ mask) as two launches: the wall kernel, then the
// pipelined stencil, which converts the wall launch's statistics (block 0); where
// the pipeline does not take the grid, the wall kernel converts them itself and
// the direct-load force (and mask) kernels follow.
static int two_launch_step(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                           void *fx, void *fy, void *fz, const void *const gradp[3], double dt, int do_mask,
                           wmibm_band_stats *stats, cudaStream_t stream)
{
    void *const f[3] = {fx, fy, fz};
    StencilConfig c;
    if (stencil_config(h, (const void *const *)tau, f, &c)) {
        int st = wall_model(h, u, v, w, tau, stats, h->logz0, stream, false);
        if (st) return st;
        if (do_mask)
            return stencil_force_mask(h, const_cast<void *>(u), const_cast<void *>(v), const_cast<void *>(w),
                                      (const void *const *)tau, f, gradp, dt, c, true, stream, stats);
        return stencil_force(h, (const void *const *)tau, f, c, stream, stats);
    }
    int st = wall_model(h, u, v, w, tau, stats, h->logz0, stream, true);
    if (st) return st;
    st = force_any(h, (const void *const *)tau, fx, fy, fz, stream);
    if (st || !do_mask) return st;
    return mask_impl(h, const_cast<void *>(u), const_cast<void *>(v), const_cast<void *>(w), gradp, dt, stream);
}

// Wall stress + force (+ mask): one cooperative launch where the pipelined
// stencil takes the grid and the tuning allows it; else returns 1 and does nothing.
static int try_fused(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *fx, void *fy, void *fz,
                     const void *const gradp[3], double dt, int do_mask, wmibm_band_stats *stats,
                     cudaStream_t stream, int *done)
{
    *done = 0;
    if (h->tuning.force_path == 3) return WMIBM_OK;
    void *const f[3] = {fx, fy, fz};
    StencilConfig c;
    if (!stencil_config(h, (const void *const *)tau, f, &c)) return WMIBM_OK;
    *done = 1;
    return stencil_step_fused(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, stream);
}

// force, then (do_mask) the body mask: one pipelined launch where the grid
// allows, else the direct-load force kernel followed by the mask kernel.
int force_mask_impl(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *fx, void *fy, void *fz,
                    const void *const gradp[3], int do_mask, double dt, bool pdl, cudaStream_t stream)
{
    void *const f[3] = {fx, fy, fz};
    StencilConfig c;
    if (stencil_config(h, (const void *const *)tau, f, &c)) {
        if (do_mask)
            return stencil_force_mask(h, u, v, w, (const void *const *)tau, f, gradp, dt, c, pdl, stream, nullptr);
        return force_any(h, (const void *const *)tau, fx, fy, fz, stream);
    }
    int st = force_any(h, (const void *const *)tau, fx, fy, fz, stream);
    if (st || !do_mask) return st;
    return mask_impl(h, u, v, w, gradp, dt, stream);
}

int mask_impl(wmibm_handle *h, void *u, void *v, void *w, const void *const gradp[3], double dt, cudaStream_t stream)
{
    if (h->dtype == WMIBM_F64) return launch<double, double>(h, u, v, w, gradp, dt, stream);
    if (h->vel_dtype == WMIBM_BF16) return launch<float, __nv_bfloat16>(h, u, v, w, gradp, dt, stream);
    return launch<float, float>(h, u, v, w, gradp, dt, stream);
}
}  // namespace wmibm

extern "C" int wmibm_mask(wmibm_handle *h, void *u, void *v, void *w, const void *const gradp[3], double dt,
                          void *stream)
{
    ApiRange nvtx_range("wmibm_mask");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w) return set_error(h, WMIBM_EINVAL, "NULL velocity pointer");
    if (gradp && (!gradp[0] || !gradp[1] || !gradp[2]))
        return set_error(h, WMIBM_EINVAL, "gradp given with a NULL component");
    if (!isfinite(dt)) return set_error(h, WMIBM_EINVAL, "dt must be finite");
    int st = check_device(h);
    if (st) return st;
    return mask_impl(h, u, v, w, gradp, dt, (cudaStream_t)stream);
}

static int check_fields(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6], void *fx,
                        void *fy, void *fz)
{
    if (!u || !v || !w || !tau || !fx || !fy || !fz)
        return set_error(h, WMIBM_EINVAL, "NULL velocity, stress or force pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    return check_device(h);
}

extern "C" int wmibm_wall_stress_force(wmibm_handle *h, const void *u, const void *v, const void *w,
                                       void *const tau[6], void *fx, void *fy, void *fz, wmibm_band_stats *stats,
                                       void *stream)
{
    ApiRange nvtx_range("wmibm_wall_stress_force");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    int st = check_fields(h, u, v, w, tau, fx, fy, fz);
    if (st) return st;
    int done = 0;
    st = try_fused(h, const_cast<void *>(u), const_cast<void *>(v), const_cast<void *>(w), tau, fx, fy, fz, nullptr,
                   0.0, 0, stats, (cudaStream_t)stream, &done);
    if (st || done) return st;
    return two_launch_step(h, u, v, w, tau, fx, fy, fz, nullptr, 0.0, 0, stats, (cudaStream_t)stream);
}

extern "C" int wmibm_force_mask(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, void *u,
                                void *v, void *w, const void *const gradp[3], double dt, void *stream)
{
    ApiRange nvtx_range("wmibm_force_mask");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    int st = check_fields(h, u, v, w, const_cast<void *const *>(tau), fx, fy, fz);
    if (st) return st;
    if (gradp && (!gradp[0] || !gradp[1] || !gradp[2]))
        return set_error(h, WMIBM_EINVAL, "gradp given with a NULL component");
    if (!isfinite(dt)) return set_error(h, WMIBM_EINVAL, "dt must be finite");
    return force_mask_impl(h, u, v, w, const_cast<void *const *>(tau), fx, fy, fz, gradp, 1, dt, false,
                           (cudaStream_t)stream);
}

extern "C" int wmibm_step(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *fx, void *fy,
                          void *fz, const void *const gradp[3], double dt, wmibm_band_stats *stats, void *stream)
{
    ApiRange nvtx_range("wmibm_step");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    int st = check_fields(h, u, v, w, tau, fx, fy, fz);
    if (st) return st;
    if (gradp && (!gradp[0] || !gradp[1] || !gradp[2]))
        return set_error(h, WMIBM_EINVAL, "gradp given with a NULL component");
    if (!isfinite(dt)) return set_error(h, WMIBM_EINVAL, "dt must be finite");
    int done = 0;
    st = try_fused(h, u, v, w, tau, fx, fy, fz, gradp, dt, 1, stats, (cudaStream_t)stream, &done);
    if (st || done) return st;
    return two_launch_step(h, u, v, w, tau, fx, fy, fz, gradp, dt, 1, stats, (cudaStream_t)stream);
}
