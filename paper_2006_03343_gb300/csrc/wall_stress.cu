// Wall model at the band nodes (Sec. 3.3 of Liu & Stevens, arXiv:2006.03343).
//
// One thread per band node: gather the 8-corner trilinear stencils of u, v
// (uv-grid) and w (w-grid) at x_c from the precomputed record, take the
// tangential part U_r = u - (u.n) n, and write the rotated log-law stress
//   tau_ij = tau_w (t_i n_j + n_i t_j),  t = U_r/|U_r|,  tau_w = -C |U_r|^2
// which is a_im a_jn tau'_mn with tau'_13 = tau'_31 = tau_w and every other
// tau'_mn = 0 (Eq. 28 and the rotation that follows it).  Extra blocks of the
// same launch zero the solid-node stresses.  Band statistics are reduced per
// warp with shuffles, per block in shared memory, and across blocks by the last
// block to finish (fixed order, so the result is deterministic).
#include "internal.cuh"

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

template <typename T>
struct RecOf;
template <>
struct RecOf<float> {
    using type = RecF32;
};
template <>
struct RecOf<double> {
    using type = RecF64;
};

struct Unpacked32 {
    float nx, ny, nz, C, ax, ay, azu, azw;
    int4 ix;
};

__device__ __forceinline__ void unpack(const RecF32 *r, int64_t t, float &nx, float &ny, float &nz, float &C,
                                       float &ax, float &ay, float &azu, float &azw, int4 &ix)
{
    const float4 a = __ldg(&r[t].nC);
    const float4 b = __ldg(&r[t].frac);
    ix = __ldg(&r[t].ix);
    nx = a.x; ny = a.y; nz = a.z; C = a.w;
    ax = b.x; ay = b.y; azu = b.z; azw = b.w;
}

__device__ __forceinline__ void unpack(const RecF64 *r, int64_t t, double &nx, double &ny, double &nz, double &C,
                                       double &ax, double &ay, double &azu, double &azw, int4 &ix)
{
    const double2 a = __ldg(&r[t].n01);
    const double2 b = __ldg(&r[t].n2C);
    const double2 c = __ldg(&r[t].fxy);
    const double2 d = __ldg(&r[t].fz);
    ix = __ldg(&r[t].ix);
    nx = a.x; ny = a.y; nz = b.x; C = b.y;
    ax = c.x; ay = c.y; azu = d.x; azw = d.y;
}

template <typename T>
__device__ __forceinline__ T lerp(T a, T b, T t) { return a + t * (b - a); }

template <typename V, typename T>
__device__ __forceinline__ T trilinear(const V *f, int64_t base, int64_t di, int64_t dj, int64_t dk, T ax, T ay,
                                       T az)
{
    const T c000 = load_vel<V, T>(f, base), c100 = load_vel<V, T>(f, base + di);
    const T c010 = load_vel<V, T>(f, base + dj), c110 = load_vel<V, T>(f, base + di + dj);
    const T c001 = load_vel<V, T>(f, base + dk), c101 = load_vel<V, T>(f, base + di + dk);
    const T c011 = load_vel<V, T>(f, base + dj + dk), c111 = load_vel<V, T>(f, base + di + dj + dk);
    const T c00 = lerp(c000, c100, ax), c10 = lerp(c010, c110, ax);
    const T c01 = lerp(c001, c101, ax), c11 = lerp(c011, c111, ax);
    return lerp(lerp(c00, c10, ay), lerp(c01, c11, ay), az);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// acc layout (kStatVals): [band][sum tau_w, sum tau_w^2, min tau_w, max U_r], band 0 = w, 1 = uv
template <typename T>
__device__ __forceinline__ void combine(T *dst, const T *src)
{
    for (int b = 0; b < 2; ++b) {
        dst[4 * b + 0] += src[4 * b + 0];
        dst[4 * b + 1] += src[4 * b + 1];
        dst[4 * b + 2] = min(dst[4 * b + 2], src[4 * b + 2]);
        dst[4 * b + 3] = max(dst[4 * b + 3], src[4 * b + 3]);
    }
}

template <typename T>
__device__ void block_reduce(T acc[kStatVals], T (*smem)[kStatVals])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = 0; b < 2; ++b) {
        acc[4 * b + 0] = warp_sum(acc[4 * b + 0]);
        acc[4 * b + 1] = warp_sum(acc[4 * b + 1]);
        acc[4 * b + 2] = warp_min(acc[4 * b + 2]);
        acc[4 * b + 3] = warp_max(acc[4 * b + 3]);
    }
    if (lane == 0)
        for (int s = 0; s < kStatVals; ++s) smem[warp][s] = acc[s];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kThreads / 32; ++w) combine(acc, smem[w]);
    __syncthreads();
}

template <typename T, typename V>
__global__ void __launch_bounds__(kThreads) k_wall_stress(WSParams<T> p)
{
    using Rec = typename RecOf<T>::type;
    __shared__ T red[kThreads / 32][kStatVals];
    __shared__ bool last;

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
    for (int b = 0; b < 2; ++b) {
        acc[4 * b + 0] = T(0);
        acc[4 * b + 1] = T(0);
        acc[4 * b + 2] = T(0);     // tau_w <= 0: 0 is the identity of the min
        acc[4 * b + 3] = T(0);     // |U_r| >= 0: 0 is the identity of the max
    }

    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t < p.nb_w + p.nb_uv) {
        const bool is_w = t < p.nb_w;
        T nx, ny, nz, C, ax, ay, azu, azw;
        int4 ix;
        unpack(reinterpret_cast<const Rec *>(p.rec), t, nx, ny, nz, C, ax, ay, azu, azw, ix);
        const int64_t di = (ix.w & 1) ? 1 - p.nx : 1;
        const int64_t dj = (ix.w & 2) ? (int64_t)(1 - p.ny) * p.nx : p.nx;
        const V *u = reinterpret_cast<const V *>(p.u);
        const V *v = reinterpret_cast<const V *>(p.v);
        const V *w = reinterpret_cast<const V *>(p.w);
        const T uc = trilinear<V, T>(u, ix.y, di, dj, p.plane, ax, ay, azu);
        const T vc = trilinear<V, T>(v, ix.y, di, dj, p.plane, ax, ay, azu);
        const T wc = trilinear<V, T>(w, ix.z, di, dj, p.plane, ax, ay, azw);
        if (p.logz0) {
            const T d = p.log_phi_c - __ldg(p.logz0 + ix.x);
            C = p.kappa2 / (d * d);
        }

        const T un = uc * nx + vc * ny + wc * nz;
        const T urx = uc - un * nx, ury = vc - un * ny, urz = wc - un * nz;
        const T ur2 = urx * urx + ury * ury + urz * urz;
        const T ur = sqrt(ur2);
        const T s = -C * ur;                      // tau_w / |U_r|
        const int32_t idx = ix.x;
        if (is_w) {
            p.txz[idx] = s * (urx * nz + nx * urz);
            p.tyz[idx] = s * (ury * nz + ny * urz);
        } else {
            p.txx[idx] = T(2) * s * (urx * nx);
            p.txy[idx] = s * (urx * ny + nx * ury);
            p.tyy[idx] = T(2) * s * (ury * ny);
            p.tzz[idx] = T(2) * s * (urz * nz);
        }
        const T tw = -C * ur2;
        const int b = is_w ? 0 : 1;
        acc[4 * b + 0] = tw;
        acc[4 * b + 1] = tw * tw;
        acc[4 * b + 2] = tw;
        acc[4 * b + 3] = ur;
    }

    if (p.stats == nullptr) return;            // uniform across the launch

    block_reduce(acc, red);
    if (threadIdx.x == 0) {
        T *dst = p.partials + (int64_t)blockIdx.x * kStatVals;
        for (int s = 0; s < kStatVals; ++s) dst[s] = acc[s];
        __threadfence();
        const unsigned prev = atomicAdd(p.ticket, 1u);
        last = (prev == p.band_blocks - 1);
    }
    __syncthreads();
    if (!last) return;

    // last band block: reduce all partials in a fixed order
    __threadfence();
    for (int b = 0; b < 2; ++b) {
        acc[4 * b + 0] = T(0);
        acc[4 * b + 1] = T(0);
        acc[4 * b + 2] = T(0);
        acc[4 * b + 3] = T(0);
    }
    for (int64_t blk = threadIdx.x; blk < p.band_blocks; blk += kThreads) {
        T src[kStatVals];
        for (int s = 0; s < kStatVals; ++s) src[s] = __ldcg(p.partials + blk * kStatVals + s);
        combine(acc, src);
    }
    block_reduce(acc, red);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            wmibm_band_stats st;
            st.count = b == 0 ? p.nb_w : p.nb_uv;
            st.sum_tw = (double)acc[4 * b + 0];
            st.sum_tw2 = (double)acc[4 * b + 1];
            st.min_tw = (double)acc[4 * b + 2];
            st.max_ur = (double)acc[4 * b + 3];
            p.stats[b] = st;
        }
        *p.ticket = 0u;                         // ready for the next call
    }
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
