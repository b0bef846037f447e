// The forcing f = -div(tau) on the vertically staggered grid (Eq. 2 and Eq. 18
// of Liu & Stevens, arXiv:2006.03343; vertical differences of Eqs. 15-16,
// horizontal derivatives by periodic second-order central differences):
//   f_x(uv k) = -[(txx[i+1]-txx[i-1])/2dx + (txy[j+1]-txy[j-1])/2dy + (txz[k+1]-txz[k])/dz]
//   f_y(uv k) = -[(txy[i+1]-txy[i-1])/2dx + (tyy[j+1]-tyy[j-1])/2dy + (tyz[k+1]-tyz[k])/dz]
//   f_z(w k)  = -[(txz[i+1]-txz[i-1])/2dx + (tyz[j+1]-tyz[j-1])/2dy + (tzz[k]-tzz[k-1])/dz]
// with f_x = f_y = 0 on the ghost uv level and f_z = 0 on the floor and lid.
//
// HBM-bound stencil: each thread owns VEC consecutive x-points of one (j) row
// and marches up a chunk of z levels, carrying txz, tyz (level k+1 -> k) and
// tzz (k -> k-1) in registers.  Centre values come in as 16-byte vector loads;
// the x-neighbours at the vector edges and the j +- 1 rows are re-read through
// L1 (they are the neighbouring threads' lines), so DRAM sees each array once.
#include "internal.cuh"

using namespace wmibm;

namespace {

template <typename T, int V>
struct Pack {
    T v[V];
};

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ldp(const T *p);

template <>
__device__ __forceinline__ Pack<float, 4> ldp<float, 4>(const float *p)
{
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    return Pack<float, 4>{{a.x, a.y, a.z, a.w}};
}
template <>
__device__ __forceinline__ Pack<float, 1> ldp<float, 1>(const float *p)
{
    return Pack<float, 1>{{__ldg(p)}};
}
template <>
__device__ __forceinline__ Pack<double, 2> ldp<double, 2>(const double *p)
{
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    return Pack<double, 2>{{a.x, a.y}};
}
template <>
__device__ __forceinline__ Pack<double, 1> ldp<double, 1>(const double *p)
{
    return Pack<double, 1>{{__ldg(p)}};
}

template <typename T, int V>
__device__ __forceinline__ void stp(T *p, const Pack<T, V> &x);
template <>
__device__ __forceinline__ void stp<float, 4>(float *p, const Pack<float, 4> &x)
{
    *reinterpret_cast<float4 *>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
template <>
__device__ __forceinline__ void stp<float, 1>(float *p, const Pack<float, 1> &x) { *p = x.v[0]; }
template <>
__device__ __forceinline__ void stp<double, 2>(double *p, const Pack<double, 2> &x)
{
    *reinterpret_cast<double2 *>(p) = make_double2(x.v[0], x.v[1]);
}
template <>
__device__ __forceinline__ void stp<double, 1>(double *p, const Pack<double, 1> &x) { *p = x.v[0]; }

template <typename T>
struct ForceParams {
    const T *txx, *txy, *tyy, *tzz, *txz, *tyz;
    T *fx, *fy, *fz;
    int32_t nx, ny, nz, kc;
    T cx, cy, cz;       // 1/(2 dx), 1/(2 dy), 1/dz
};

template <typename T, int V>
__global__ void __launch_bounds__(256, 3) k_force(ForceParams<T> p)
{
    const int32_t nq = p.nx / V;
    const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t j = blockIdx.y * blockDim.y + threadIdx.y;
    if (q >= nq || j >= p.ny) return;
    const int32_t k0 = blockIdx.z * p.kc;
    const int32_t k1 = min(k0 + p.kc, p.nz);

    const int32_t i = q * V;
    const int32_t im = (i == 0) ? p.nx - 1 : i - 1;
    const int32_t ip = (i + V == p.nx) ? 0 : i + V;
    const int32_t jm = (j == 0) ? p.ny - 1 : j - 1;
    const int32_t jp = (j + 1 == p.ny) ? 0 : j + 1;
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int64_t row = (int64_t)j * p.nx, rowm = (int64_t)jm * p.nx, rowp = (int64_t)jp * p.nx;

    int64_t ob = (int64_t)k0 * plane;
    Pack<T, V> xz_k = ldp<T, V>(p.txz + ob + row + i);
    Pack<T, V> yz_k = ldp<T, V>(p.tyz + ob + row + i);
    Pack<T, V> zz_km;
    for (int e = 0; e < V; ++e) zz_km.v[e] = T(0);
    if (k0 > 0) zz_km = ldp<T, V>(p.tzz + ob - plane + row + i);

    for (int32_t k = k0; k < k1; ++k, ob += plane) {
        const int64_t o = ob + row + i;
        const bool top = (k == p.nz - 1);
        const Pack<T, V> xx = ldp<T, V>(p.txx + o);
        const T xxl = __ldg(p.txx + ob + row + im), xxr = __ldg(p.txx + ob + row + ip);
        const Pack<T, V> xy = ldp<T, V>(p.txy + o);
        const T xyl = __ldg(p.txy + ob + row + im), xyr = __ldg(p.txy + ob + row + ip);
        const Pack<T, V> xyjm = ldp<T, V>(p.txy + ob + rowm + i), xyjp = ldp<T, V>(p.txy + ob + rowp + i);
        const Pack<T, V> yyjm = ldp<T, V>(p.tyy + ob + rowm + i), yyjp = ldp<T, V>(p.tyy + ob + rowp + i);
        const Pack<T, V> yzjm = ldp<T, V>(p.tyz + ob + rowm + i), yzjp = ldp<T, V>(p.tyz + ob + rowp + i);
        const T xzl = __ldg(p.txz + ob + row + im), xzr = __ldg(p.txz + ob + row + ip);
        const Pack<T, V> zz = ldp<T, V>(p.tzz + o);
        Pack<T, V> xz_kp, yz_kp;
        if (!top) {
            xz_kp = ldp<T, V>(p.txz + o + plane);
            yz_kp = ldp<T, V>(p.tyz + o + plane);
        } else {
            xz_kp = xz_k;
            yz_kp = yz_k;
        }

        Pack<T, V> Fx, Fy, Fz;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const T xxm = e == 0 ? xxl : xx.v[e - 1], xxp = e == V - 1 ? xxr : xx.v[e + 1];
            const T xym = e == 0 ? xyl : xy.v[e - 1], xyp = e == V - 1 ? xyr : xy.v[e + 1];
            const T xzm = e == 0 ? xzl : xz_k.v[e - 1], xzp = e == V - 1 ? xzr : xz_k.v[e + 1];
            const T fx = -((xxp - xxm) * p.cx + (xyjp.v[e] - xyjm.v[e]) * p.cy + (xz_kp.v[e] - xz_k.v[e]) * p.cz);
            const T fy = -((xyp - xym) * p.cx + (yyjp.v[e] - yyjm.v[e]) * p.cy + (yz_kp.v[e] - yz_k.v[e]) * p.cz);
            const T fz = -((xzp - xzm) * p.cx + (yzjp.v[e] - yzjm.v[e]) * p.cy + (zz.v[e] - zz_km.v[e]) * p.cz);
            Fx.v[e] = top ? T(0) : fx;
            Fy.v[e] = top ? T(0) : fy;
            Fz.v[e] = (top || k == 0) ? T(0) : fz;
        }
        stp<T, V>(p.fx + o, Fx);
        stp<T, V>(p.fy + o, Fy);
        stp<T, V>(p.fz + o, Fz);
        xz_k = xz_kp;
        yz_k = yz_kp;
        zz_km = zz;
    }
}

template <typename T, int V>
int launch(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream, int bx,
           int by, int kc)
{
    ForceParams<T> p;
    p.txx = (const T *)tau[0]; p.txy = (const T *)tau[1]; p.tyy = (const T *)tau[2];
    p.tzz = (const T *)tau[3]; p.txz = (const T *)tau[4]; p.tyz = (const T *)tau[5];
    p.fx = (T *)fx; p.fy = (T *)fy; p.fz = (T *)fz;
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz; p.kc = kc;
    p.cx = (T)(1.0 / (2.0 * h->dx));
    p.cy = (T)(1.0 / (2.0 * h->dy));
    p.cz = (T)(1.0 / h->dz);
    const int nq = h->nx / V;
    if (bx > nq) bx = nq;
    if (bx * by > 256) by = 256 / bx;
    if (by < 1) by = 1;
    dim3 block(bx, by, 1);
    dim3 grid((nq + bx - 1) / bx, (h->ny + by - 1) / by, (h->nz + kc - 1) / kc);
    if (grid.y > 65535 || grid.z > 65535) return set_error(h, WMIBM_EINVAL, "grid too large for the force launch");
    k_force<T, V><<<grid, block, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_force launch");
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace wmibm {

// Tile of the force launch: bx vectors along x, by rows, kc levels per thread.
int force_impl(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream, int bx,
               int by, int kc)
{
    if (kc < 1) kc = 1;
    bool al = aligned16(fx) && aligned16(fy) && aligned16(fz);
    for (int c = 0; c < 6; ++c) al = al && aligned16(tau[c]);
    if (h->dtype == WMIBM_F64) {
        if (al && h->nx % 2 == 0) return launch<double, 2>(h, tau, fx, fy, fz, stream, bx, by, kc);
        return launch<double, 1>(h, tau, fx, fy, fz, stream, bx, by, kc);
    }
    if (al && h->nx % 4 == 0) return launch<float, 4>(h, tau, fx, fy, fz, stream, bx, by, kc);
    return launch<float, 1>(h, tau, fx, fy, fz, stream, bx, by, kc);
}

void force_default_tile(const wmibm_handle *h, int *bx, int *by, int *kc)
{
    *bx = h->tuning.direct_bx > 0 ? h->tuning.direct_bx : 32;
    *by = h->tuning.direct_by > 0 ? h->tuning.direct_by : 8;
    *kc = h->tuning.direct_kc > 0 ? h->tuning.direct_kc : 4;
}

bool stencil_config(const wmibm_handle *h, const void *const tau[6], void *const f[3], StencilConfig *out);
int stencil_force(wmibm_handle *h, const void *const tau[6], void *const f[3], const StencilConfig &c,
                  cudaStream_t stream, wmibm_band_stats *emit);

// f = -div(tau): the bulk-copy pipeline where it applies, else the direct-load kernel.
int force_any(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream)
{
    void *const f[3] = {fx, fy, fz};
    StencilConfig c;
    if (stencil_config(h, tau, f, &c)) return stencil_force(h, tau, f, c, stream, nullptr);
    int bx, by, kc;
    force_default_tile(h, &bx, &by, &kc);
    return force_impl(h, tau, fx, fy, fz, stream, bx, by, kc);
}

}  // namespace wmibm

extern "C" int wmibm_force(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, void *stream)
{
    ApiRange nvtx_range("wmibm_force");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!tau || !fx || !fy || !fz) return set_error(h, WMIBM_EINVAL, "NULL stress or force pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    int st = check_device(h);
    if (st) return st;
    return force_any(h, tau, fx, fy, fz, (cudaStream_t)stream);
}
