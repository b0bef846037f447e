// The wall model at one band node (Sec. 3.3 of Liu & Stevens, arXiv:2006.03343),
// shared by the stand-alone wall-stress kernel and the fused stencil kernel so
// that both produce identical values.
//
//   u_c  = trilinear(u, v on the uv-grid; w on the w-grid) at x_c
//   U_r  = u_c - (u_c . n) n,  s = -C |U_r|
//   tau_ij = s (U_r,i n_j + n_i U_r,j)    (= a_im a_jn tau'_mn, tau'_13 = tau'_31 = tau_w)
//   tau_w  = -C |U_r|^2                    (Eq. 28, C = kappa^2 / ln^2(phi_c / z0))
#pragma once

#include "internal.cuh"

namespace wmibm {

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

// Result of the wall model at one band node.
template <typename T>
struct BandOut {
    int32_t idx;      // node index
    T t0, t1, t2, t3; // w-band: (txz, tyz, -, -); uv-band: (txx, txy, tyy, tzz)
    T tw, ur;         // tau_w and |U_r|
};

// Inputs of the wall model at one band node: the record and the 8 corner
// values of each velocity component (corner c: bit 0 = +x, bit 1 = +y, bit 2 = +z).
template <typename T>
struct BandIn {
    T n0, n1, n2, C, ax, ay, azu, azw;
    int32_t idx;
    T cu[8], cv[8], cw[8];
};

// Loads record t and its 24 corner values (all loads independent of each
// other once the record is in, so that callers can have several nodes' loads
// in flight before any arithmetic).
template <typename T, typename V>
__device__ __forceinline__ void band_gather(const int4 ix, const V *u, const V *v, const V *w, int32_t nx,
                                            int32_t ny, int64_t plane, BandIn<T> &b);

template <typename T, typename V>
__device__ __forceinline__ void band_fetch(const void *rec, int64_t t, const V *u, const V *v, const V *w,
                                           int32_t nx, int32_t ny, int64_t plane, BandIn<T> &b)
{
    using Rec = typename RecOf<T>::type;
    int4 ix;
    unpack(reinterpret_cast<const Rec *>(rec), t, b.n0, b.n1, b.n2, b.C, b.ax, b.ay, b.azu, b.azw, ix);
    band_gather<T, V>(ix, u, v, w, nx, ny, plane, b);
}

// The same from a copy of the record in shared memory.
__device__ __forceinline__ void unpack_shared(const RecF32 *r, float &nx, float &ny, float &nz, float &C, float &ax,
                                              float &ay, float &azu, float &azw, int4 &ix)
{
    const float4 a = r->nC, b = r->frac;
    ix = r->ix;
    nx = a.x; ny = a.y; nz = a.z; C = a.w;
    ax = b.x; ay = b.y; azu = b.z; azw = b.w;
}
__device__ __forceinline__ void unpack_shared(const RecF64 *r, double &nx, double &ny, double &nz, double &C,
                                              double &ax, double &ay, double &azu, double &azw, int4 &ix)
{
    const double2 a = r->n01, b = r->n2C, c = r->fxy, d = r->fz;
    ix = r->ix;
    nx = a.x; ny = a.y; nz = b.x; C = b.y;
    ax = c.x; ay = c.y; azu = d.x; azw = d.y;
}

template <typename T, typename V>
__device__ __forceinline__ void band_fetch_shared(const typename RecOf<T>::type *srec, const V *u, const V *v,
                                                  const V *w, int32_t nx, int32_t ny, int64_t plane, BandIn<T> &b)
{
    int4 ix;
    unpack_shared(srec, b.n0, b.n1, b.n2, b.C, b.ax, b.ay, b.azu, b.azw, ix);
    band_gather<T, V>(ix, u, v, w, nx, ny, plane, b);
}

// The 24 corner values of the node whose record unpacked to ix.
template <typename T, typename V>
__device__ __forceinline__ void band_gather(const int4 ix, const V *u, const V *v, const V *w, int32_t nx,
                                            int32_t ny, int64_t plane, BandIn<T> &b)
{
    // 32-bit index arithmetic: a grid has fewer than 2^31 nodes (checked at init)
    // and every corner is one of its nodes, so one multiply-add forms each address
    b.idx = ix.x;
    const int32_t di = (ix.w & 1) ? 1 - nx : 1;
    const int32_t dj = (ix.w & 2) ? (1 - ny) * nx : nx;
    const int32_t dk = (int32_t)plane;
    const V *const pu = u + ix.y, *const pv = v + ix.y, *const pw = w + ix.z;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int32_t o = ((c & 1) ? di : 0) + ((c & 2) ? dj : 0) + ((c & 4) ? dk : 0);
        b.cu[c] = load_vel<V, T>(pu, o);
        b.cv[c] = load_vel<V, T>(pv, o);
        b.cw[c] = load_vel<V, T>(pw, o);
    }
}

template <typename T>
__device__ __forceinline__ T trilinear8(const T *c, T ax, T ay, T az)
{
    const T c00 = lerp(c[0], c[1], ax), c10 = lerp(c[2], c[3], ax);
    const T c01 = lerp(c[4], c[5], ax), c11 = lerp(c[6], c[7], ax);
    return lerp(lerp(c00, c10, ay), lerp(c01, c11, ay), az);
}

// The wall model of a fetched node (t < nb_w: a w-band node, else uv-band).
template <typename T>
__device__ __forceinline__ BandOut<T> band_finish(const BandIn<T> &b, bool is_w, const T *logz0, T log_phi_c,
                                                  T kappa2)
{
    const T nxv = b.n0, nyv = b.n1, nzv = b.n2;
    T C = b.C;
    const T uc = trilinear8(b.cu, b.ax, b.ay, b.azu);
    const T vc = trilinear8(b.cv, b.ax, b.ay, b.azu);
    const T wc = trilinear8(b.cw, b.ax, b.ay, b.azw);
    if (logz0) {
        const T d = log_phi_c - __ldg(logz0 + b.idx);
        C = kappa2 / (d * d);
    }
    const T un = uc * nxv + vc * nyv + wc * nzv;
    const T urx = uc - un * nxv, ury = vc - un * nyv, urz = wc - un * nzv;
    const T ur2 = urx * urx + ury * ury + urz * urz;
    const T ur = sqrt(ur2);
    const T s = -C * ur;
    BandOut<T> o;
    o.idx = b.idx;
    if (is_w) {
        o.t0 = s * (urx * nzv + nxv * urz);
        o.t1 = s * (ury * nzv + nyv * urz);
        o.t2 = T(0);
        o.t3 = T(0);
    } else {
        o.t0 = T(2) * s * (urx * nxv);
        o.t1 = s * (urx * nyv + nxv * ury);
        o.t2 = T(2) * s * (ury * nyv);
        o.t3 = T(2) * s * (urz * nzv);
    }
    o.tw = -C * ur2;
    o.ur = ur;
    return o;
}

// Evaluates the wall model for record t (t < nb_w: a w-band node, else a uv-band node).
template <typename T, typename V>
__device__ __forceinline__ BandOut<T> band_model(const void *rec, int64_t t, bool is_w, const V *u, const V *v,
                                                 const V *w, int32_t nx, int32_t ny, int64_t plane, const T *logz0,
                                                 T log_phi_c, T kappa2)
{
    BandIn<T> b;
    band_fetch<T, V>(rec, t, u, v, w, nx, ny, plane, b);
    return band_finish<T>(b, is_w, logz0, log_phi_c, kappa2);
}

// ------------------------------------------------------------------------- //
// band statistics reduction: warp shuffles, shared memory, then the last block
// acc layout: [band][sum tau_w, sum tau_w^2, min tau_w, max U_r], band 0 = w, 1 = uv
// ------------------------------------------------------------------------- //
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

template <typename T>
__device__ __forceinline__ void stats_identity(T *acc)
{
    for (int s = 0; s < kStatVals; ++s) acc[s] = T(0);   // tau_w <= 0 and |U_r| >= 0: 0 is the identity
}

// (constant indices only, so that acc stays in registers)
template <typename T>
__device__ __forceinline__ void stats_add(T *acc, int b, T tw, T ur)
{
    if (b == 0) {
        acc[0] += tw;
        acc[1] += tw * tw;
        acc[2] = min(acc[2], tw);
        acc[3] = max(acc[3], ur);
    } else {
        acc[4] += tw;
        acc[5] += tw * tw;
        acc[6] = min(acc[6], tw);
        acc[7] = max(acc[7], ur);
    }
}

template <typename T>
__device__ __forceinline__ void stats_combine(T *dst, const T *src)
{
    for (int b = 0; b < 2; ++b) {
        dst[4 * b + 0] += src[4 * b + 0];
        dst[4 * b + 1] += src[4 * b + 1];
        dst[4 * b + 2] = min(dst[4 * b + 2], src[4 * b + 2]);
        dst[4 * b + 3] = max(dst[4 * b + 3], src[4 * b + 3]);
    }
}

// All threads of the block call this; thread 0 ends up with the block total.
template <typename T>
__device__ void stats_block_reduce(T acc[kStatVals], T (*smem)[kStatVals])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
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
        for (int w = 1; w < nwarps; ++w) stats_combine(acc, smem[w]);
    __syncthreads();
}

// Every block of the launch that takes part calls this with its reduced
// partial in thread 0's acc; the last block to arrive writes stats[0..1]
// (counts from the handle) and re-arms the ticket.  smem must hold 32 rows.
template <typename T>
__device__ void stats_finish(T acc[kStatVals], T (*smem)[kStatVals], T *partials, unsigned *ticket,
                             unsigned nblocks, wmibm_band_stats *stats, int64_t count_w, int64_t count_uv,
                             int64_t nzc_w, int64_t nzc_uv)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        T *dst = partials + (int64_t)blockIdx.x * kStatVals;
        for (int s = 0; s < kStatVals; ++s) dst[s] = acc[s];
        __threadfence();
        const unsigned prev = atomicAdd(ticket, 1u);
        last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    stats_identity(acc);
    for (int64_t blk = threadIdx.x; blk < nblocks; blk += blockDim.x) {
        T src[kStatVals];
        for (int s = 0; s < kStatVals; ++s) src[s] = __ldcg(partials + blk * kStatVals + s);
        stats_combine(acc, src);
    }
    stats_block_reduce(acc, smem);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            wmibm_band_stats st;
            st.count = b == 0 ? count_w : count_uv;
            st.n_zclamped = b == 0 ? nzc_w : nzc_uv;
            st.sum_tw = (double)acc[4 * b + 0];
            st.sum_tw2 = (double)acc[4 * b + 1];
            st.min_tw = (double)acc[4 * b + 2];
            st.max_ur = (double)acc[4 * b + 3];
            stats[b] = st;
        }
        *ticket = 0u;
    }
}

// Order-preserving encoding of a non-negative value for 64-bit integer atomics.
__device__ __forceinline__ unsigned long long ordered_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x > 0.0 ? x : 0.0);
}

// Adds one block's reduced statistics (thread 0's acc) to the FP64 accumulator
// sacc[8] = per band (sum tau_w, sum tau_w^2, bits of -min tau_w, bits of max
// |U_r|) with fire-and-forget reductions (no fence, no wait).
template <typename T>
__device__ __forceinline__ void stats_red(const T acc[kStatVals], double *sacc)
{
    for (int b = 0; b < 2; ++b) {
        atomicAdd(sacc + 4 * b + 0, (double)acc[4 * b + 0]);
        atomicAdd(sacc + 4 * b + 1, (double)acc[4 * b + 1]);
        atomicMax(reinterpret_cast<unsigned long long *>(sacc + 4 * b + 2), ordered_bits(-(double)acc[4 * b + 2]));
        atomicMax(reinterpret_cast<unsigned long long *>(sacc + 4 * b + 3), ordered_bits((double)acc[4 * b + 3]));
    }
}

// Converts the accumulator into wmibm_band_stats[2] and clears it for the next
// call.  One thread, after every contribution is complete and visible.
__device__ __forceinline__ void stats_emit(double *sacc, wmibm_band_stats *stats, int64_t count_w, int64_t count_uv,
                                           int64_t nzc_w, int64_t nzc_uv)
{
    for (int b = 0; b < 2; ++b) {
        wmibm_band_stats st;
        st.count = b == 0 ? count_w : count_uv;
        st.n_zclamped = b == 0 ? nzc_w : nzc_uv;
        st.sum_tw = __ldcg(sacc + 4 * b + 0);
        st.sum_tw2 = __ldcg(sacc + 4 * b + 1);
        st.min_tw = -__longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(sacc + 4 * b + 2)));
        st.max_ur = __longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(sacc + 4 * b + 3)));
        if (st.min_tw == 0.0) st.min_tw = 0.0;   // no -0 for an empty band
        stats[b] = st;
        for (int q = 0; q < 4; ++q) sacc[4 * b + q] = 0.0;
    }
}

}  // namespace wmibm
