// The Smagorinsky sub-grid stress with Mason's wall damping (Eqs. 4-7 of Liu &
// Stevens, arXiv:2006.03343) at the fluid nodes:
//   tau_ij = -2 nu_t S_ij,  S = (grad u + grad u^T)/2,  nu_t = lambda^2 |S|,
//   |S| = sqrt(2 S:S),  1/lambda^2 = 1/lambda_0^2 + 1/[kappa (z + z0)]^2,
//   lambda_0 = C_s (dx dy dz)^(1/3),
// with z the node's distance phi above the immersed surface.  Each component
// sits on its own node: S11, S22, S12 (periodic central differences) and S33
// (the w-levels above and below, Eq. 16) on uv-nodes; S13, S23 on w-nodes (the
// uv-levels below and above, Eq. 15).  |S| on a uv-node averages S13, S23 of
// the w-levels below and above it (the floor repeats the level above it, the
// stress-free lid contributes 0); on a w-node it averages S11, S22, S33, S12 of
// the uv-levels below and above it.  Band and solid entries (the wall model's),
// the ghost uv-level and the floor w-level are left as they are; the lid's
// fluid tau_xz, tau_yz become 0 (Eq. 10).
//
// One thread per column (i, j) marches up a chunk of levels, forming each
// level's uv strain and w shear once; x and y neighbours come through L1, so
// DRAM sees each velocity array and wall-term array once and the stress arrays
// once.
#include <math.h>
#include <stdlib.h>

#include "internal.cuh"

using namespace wmibm;

namespace {

template <typename T, typename V>
struct SgsParams {
    const V *u, *v, *w;
    const T *wt_uv, *wt_w;      // 1/[kappa (phi + z0)]^2 at fluid nodes, -1 at band, -2 at solid nodes
    T *txx, *txy, *tyy, *tzz, *txz, *tyz;
    int32_t nx, ny, nz;
    T cx, cy, rdz;              // 1/(2 dx), 1/(2 dy), 1/dz
    T inv_lam0_sq;              // 1/lambda_0^2
};

template <typename T, typename V>
struct Field {
    const V *p;
    int32_t nx, ny;
    int64_t plane;
    __device__ __forceinline__ T at(int i, int j, int k) const
    {
        return load_vel<V, T>(p, (int64_t)k * plane + (int64_t)j * nx + i);
    }
};

// The strain of uv-level k at column (i, j): S11, S22, S12 (periodic central
// differences) and S33 (Eq. 16), for 0 <= k <= nz-2.
template <typename T>
struct Uv {
    T s11, s22, s12, s33;
};
// The shear of w-level k at column (i, j): S13, S23 (Eq. 15) for 1 <= k <= nz-2;
// the floor repeats level 1, the lid is 0.
template <typename T>
struct Ws {
    T s13, s23;
};

template <typename T, typename V>
struct Column {
    Field<T, V> U, Vf, W;
    int i, j, im, ip, jm, jp, nz;
    T cx, cy, rdz;

    __device__ __forceinline__ Uv<T> uv(int k) const
    {
        Uv<T> a;
        a.s11 = (U.at(ip, j, k) - U.at(im, j, k)) * cx;
        a.s22 = (Vf.at(i, jp, k) - Vf.at(i, jm, k)) * cy;
        a.s12 = T(0.5) * ((U.at(i, jp, k) - U.at(i, jm, k)) * cy + (Vf.at(ip, j, k) - Vf.at(im, j, k)) * cx);
        a.s33 = (W.at(i, j, k + 1) - W.at(i, j, k)) * rdz;
        return a;
    }
    __device__ __forceinline__ Ws<T> ws(int k) const
    {
        if (k >= nz - 1) return Ws<T>{T(0), T(0)};
        if (k == 0) k = 1;
        Ws<T> b;
        b.s13 = T(0.5) * ((U.at(i, j, k) - U.at(i, j, k - 1)) * rdz + (W.at(ip, j, k) - W.at(im, j, k)) * cx);
        b.s23 = T(0.5) * ((Vf.at(i, j, k) - Vf.at(i, j, k - 1)) * rdz + (W.at(i, jp, k) - W.at(i, jm, k)) * cy);
        return b;
    }
};

// Stress of a fluid uv-node from its level's strain and the shear of the w-levels below
// and above it: (txx, tyy, tzz, txy) = -2 lambda^2 |S| (S11, S22, S33, S12).
template <typename T>
__device__ __forceinline__ void uv_stress(const Uv<T> &a, const Ws<T> &lo, const Ws<T> &hi, T wt, T inv_lam0_sq,
                                          T out[4])
{
    const T s13 = T(0.5) * (lo.s13 + hi.s13), s23 = T(0.5) * (lo.s23 + hi.s23);
    const T mag = sqrt(T(2) * (a.s11 * a.s11 + a.s22 * a.s22 + a.s33 * a.s33) +
                       T(4) * (a.s12 * a.s12 + s13 * s13 + s23 * s23));
    const T nu2 = T(-2) * mag / (inv_lam0_sq + wt);          // -2 lambda^2 |S|
    out[0] = nu2 * a.s11;
    out[1] = nu2 * a.s22;
    out[2] = nu2 * a.s33;
    out[3] = nu2 * a.s12;
}

// Stress of a fluid interior w-node from its shear and the strain of the uv-levels
// below and above it: (txz, tyz) = -2 lambda^2 |S| (S13, S23).
template <typename T>
__device__ __forceinline__ void w_stress(const Uv<T> &lo, const Uv<T> &hi, const Ws<T> &b, T wt, T inv_lam0_sq,
                                         T out[2])
{
    const T a11 = T(0.5) * (lo.s11 + hi.s11), a22 = T(0.5) * (lo.s22 + hi.s22);
    const T a12 = T(0.5) * (lo.s12 + hi.s12), a33 = T(0.5) * (lo.s33 + hi.s33);
    const T mag = sqrt(T(2) * (a11 * a11 + a22 * a22 + a33 * a33) + T(4) * (a12 * a12 + b.s13 * b.s13 + b.s23 * b.s23));
    const T nu2 = T(-2) * mag / (inv_lam0_sq + wt);
    out[0] = nu2 * b.s13;
    out[1] = nu2 * b.s23;
}

// The velocity values of level L that, with the centre values of level L-1 and
// w(L), form the uv strain of level L and the w shear of level L.
template <typename T>
struct Raw {
    T u_ip, u_im, u_jp, u_jm, v_ip, v_im, v_jp, v_jm;  // horizontal neighbours on level L
    T u_c, v_c;                                         // u, v at (i, j, L)
    T w_up;                                             // w at (i, j, L+1)
    T w_ip, w_im, w_jp, w_jm;                           // w neighbours on level L
};

template <typename T, typename V>
__device__ __forceinline__ Raw<T> load_raw(const Column<T, V> &c, int L)
{
    Raw<T> r;
    if (L <= c.nz - 2) {
        r.u_ip = c.U.at(c.ip, c.j, L); r.u_im = c.U.at(c.im, c.j, L);
        r.u_jp = c.U.at(c.i, c.jp, L); r.u_jm = c.U.at(c.i, c.jm, L);
        r.v_ip = c.Vf.at(c.ip, c.j, L); r.v_im = c.Vf.at(c.im, c.j, L);
        r.v_jp = c.Vf.at(c.i, c.jp, L); r.v_jm = c.Vf.at(c.i, c.jm, L);
        r.u_c = c.U.at(c.i, c.j, L); r.v_c = c.Vf.at(c.i, c.j, L);
        r.w_up = c.W.at(c.i, c.j, L + 1);
        r.w_ip = c.W.at(c.ip, c.j, L); r.w_im = c.W.at(c.im, c.j, L);
        r.w_jp = c.W.at(c.i, c.jp, L); r.w_jm = c.W.at(c.i, c.jm, L);
    } else {
        r = Raw<T>{};
    }
    return r;
}

// One thread per column (i, j) marching up a chunk of kc levels: each level's uv
// strain and w shear are formed once and reused by the uv-node above/below and
// the w-node between them.  Software-pipelined: the loads of level k+2 are in
// flight while level k+1's strain and level k's stresses are formed.
template <typename T, typename V>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_sgs(SgsParams<T, V> p, int kc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(k0 + kc, p.nz);
    const int64_t plane = (int64_t)p.nx * p.ny;
    Column<T, V> c;
    c.U = Field<T, V>{p.u, p.nx, p.ny, plane};
    c.Vf = Field<T, V>{p.v, p.nx, p.ny, plane};
    c.W = Field<T, V>{p.w, p.nx, p.ny, plane};
    c.i = i; c.j = j;
    c.im = i == 0 ? p.nx - 1 : i - 1; c.ip = i + 1 == p.nx ? 0 : i + 1;
    c.jm = j == 0 ? p.ny - 1 : j - 1; c.jp = j + 1 == p.ny ? 0 : j + 1;
    c.nz = p.nz; c.cx = p.cx; c.cy = p.cy; c.rdz = p.rdz;

    Uv<T> a_prev = k0 >= 1 ? c.uv(k0 - 1) : Uv<T>{0, 0, 0, 0};
    Uv<T> a_cur = k0 <= p.nz - 2 ? c.uv(k0) : Uv<T>{0, 0, 0, 0};
    Ws<T> b_cur = c.ws(k0);
    // carried centre values of level k0 and w(k0+1), then the raw values of level k0+1
    T u_c = k0 <= p.nz - 2 ? c.U.at(i, j, k0) : T(0);
    T v_c = k0 <= p.nz - 2 ? c.Vf.at(i, j, k0) : T(0);
    T w_c = k0 <= p.nz - 2 ? c.W.at(i, j, k0 + 1) : T(0);
    Raw<T> raw = load_raw(c, k0 + 1);
    int64_t o = (int64_t)k0 * plane + (int64_t)j * p.nx + i;
    for (int k = k0; k < k1; ++k, o += plane) {
        const Raw<T> nxt = load_raw(c, k + 2);                      // in flight during this level
        const T wt_uv = k <= p.nz - 2 ? p.wt_uv[o] : T(-1);
        const T wt_w = k >= 1 ? p.wt_w[o] : T(-1);
        // level k+1 from the raw values: uv strain (valid up to nz-2) and w shear (lid 0)
        const int L = k + 1;
        Uv<T> a_next{0, 0, 0, 0};
        Ws<T> b_next{0, 0};
        if (L <= p.nz - 2) {
            a_next.s11 = (raw.u_ip - raw.u_im) * p.cx;
            a_next.s22 = (raw.v_jp - raw.v_jm) * p.cy;
            a_next.s12 = T(0.5) * ((raw.u_jp - raw.u_jm) * p.cy + (raw.v_ip - raw.v_im) * p.cx);
            a_next.s33 = (raw.w_up - w_c) * p.rdz;
            b_next.s13 = T(0.5) * ((raw.u_c - u_c) * p.rdz + (raw.w_ip - raw.w_im) * p.cx);
            b_next.s23 = T(0.5) * ((raw.v_c - v_c) * p.rdz + (raw.w_jp - raw.w_jm) * p.cy);
        }
        if (wt_uv >= T(0)) {                                        // uv-node (i, j, k)
            T t[4];
            uv_stress(a_cur, b_cur, b_next, wt_uv, p.inv_lam0_sq, t);
            p.txx[o] = t[0];
            p.tyy[o] = t[1];
            p.tzz[o] = t[2];
            p.txy[o] = t[3];
        }
        if (wt_w >= T(0)) {                                         // w-node (i, j, k); the floor is left
            T t[2] = {T(0), T(0)};                                  // the lid: no stress (Eq. 10)
            if (k < p.nz - 1) w_stress(a_prev, a_cur, b_cur, wt_w, p.inv_lam0_sq, t);
            p.txz[o] = t[0];
            p.tyz[o] = t[1];
        }
        a_prev = a_cur;
        a_cur = a_next;
        b_cur = b_next;
        u_c = raw.u_c;
        v_c = raw.v_c;
        w_c = raw.w_up;
        raw = nxt;
    }
}

// ---------------------------------------------------------------------------
// The stress and the forcing in one pass.  A block owns a tile of TX x TY output
// columns and one column of halo around it: each of its (TX+2) x (TY+2) threads
// marches one column up a chunk of levels, forms the stress of its uv-node and
// w-node on every level -- the Smagorinsky stress at fluid nodes, the wall
// model's value (read from tau) at band nodes, 0 at solid nodes, the caller's
// value on the floor w-level -- and leaves the level in shared memory; the
// interior threads then form f = -div tau (Eq. 2 / Eq. 18, Eqs. 15-16) with the
// operations of the central-difference force kernel.  The stress arrays are only
// read (band nodes and the floor), never written.
constexpr int kFuseX = 32, kFuseY = 8;          // threads per block: tile plus halo
constexpr int kFuseLevels = 16;                 // levels per block

template <typename T, typename V>
struct FuseParams {
    SgsParams<T, V> s;
    T *fx, *fy, *fz;
    T cz;                                       // 1/dz of the divergence
};

template <typename T, typename V>
__device__ __forceinline__ void node_uv(const FuseParams<T, V> &p, const Column<T, V> &c, int k, int64_t o,
                                        const Uv<T> &a, const Ws<T> &lo, const Ws<T> &hi, T out[4])
{
    const T wt = p.s.wt_uv[o];
    if (wt >= T(0)) {
        uv_stress(a, lo, hi, wt, p.s.inv_lam0_sq, out);
    } else if (wt > T(-1.5)) {                  // band: the wall model's stress
        out[0] = p.s.txx[o];
        out[1] = p.s.tyy[o];
        out[2] = p.s.tzz[o];
        out[3] = p.s.txy[o];
    } else {
        out[0] = out[1] = out[2] = out[3] = T(0);
    }
}

template <typename T, typename V>
__device__ __forceinline__ void node_w(const FuseParams<T, V> &p, int k, int64_t o, const Uv<T> &lo, const Uv<T> &hi,
                                       const Ws<T> &b, T out[2])
{
    const T wt = p.s.wt_w[o];
    if (wt < T(-1.5)) {                         // solid
        out[0] = out[1] = T(0);
    } else if (wt < T(0) || k == 0) {           // band, or the floor level: the values given
        out[0] = p.s.txz[o];
        out[1] = p.s.tyz[o];
    } else if (k == p.s.nz - 1) {               // fluid lid: no stress
        out[0] = out[1] = T(0);
    } else {
        w_stress(lo, hi, b, wt, p.s.inv_lam0_sq, out);
    }
}

template <typename T, typename V>
__global__ void __launch_bounds__(kFuseX * kFuseY) k_sgs_force(FuseParams<T, V> p)
{
    __shared__ T sxx[kFuseY][kFuseX], sxy[kFuseY][kFuseX], syy[kFuseY][kFuseX];
    __shared__ T sxz[kFuseY][kFuseX], syz[kFuseY][kFuseX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = p.s.nx, ny = p.s.ny, nz = p.s.nz;
    const int ci = blockIdx.x * (kFuseX - 2) - 1 + tx;          // this thread's column, before wrapping
    const int cj = blockIdx.y * (kFuseY - 2) - 1 + ty;
    const int i = ((ci % nx) + nx) % nx, j = ((cj % ny) + ny) % ny;
    const bool out_col = tx >= 1 && tx <= kFuseX - 2 && ty >= 1 && ty <= kFuseY - 2 && ci < nx && cj < ny;
    const int64_t plane = (int64_t)nx * ny;
    Column<T, V> c;
    c.U = Field<T, V>{p.s.u, nx, ny, plane};
    c.Vf = Field<T, V>{p.s.v, nx, ny, plane};
    c.W = Field<T, V>{p.s.w, nx, ny, plane};
    c.i = i; c.j = j;
    c.im = i == 0 ? nx - 1 : i - 1; c.ip = i + 1 == nx ? 0 : i + 1;
    c.jm = j == 0 ? ny - 1 : j - 1; c.jp = j + 1 == ny ? 0 : j + 1;
    c.nz = nz; c.cx = p.s.cx; c.cy = p.s.cy; c.rdz = p.s.rdz;
    const Uv<T> zero_uv{0, 0, 0, 0};

    const int k0 = blockIdx.z * kFuseLevels;
    const int k1 = min(k0 + kFuseLevels, nz);
    const int64_t col = (int64_t)j * nx + i;
    // state entering level k: the strain of uv-level k and the shear of w-level k,
    // the stress of w-node k and the tzz of uv-node k-1
    Uv<T> a_k = k0 <= nz - 2 ? c.uv(k0) : zero_uv;
    Ws<T> b_k = c.ws(k0);
    T wk[2];
    {
        const Uv<T> a_m = k0 >= 1 ? c.uv(k0 - 1) : zero_uv;
        node_w(p, k0, (int64_t)k0 * plane + col, a_m, a_k, b_k, wk);
    }
    T zz_m = T(0);
    if (k0 >= 1) {
        const Uv<T> a_m = c.uv(k0 - 1);
        T t[4];
        node_uv(p, c, k0 - 1, (int64_t)(k0 - 1) * plane + col, a_m, c.ws(k0 - 1), b_k, t);
        zz_m = t[2];
    }
    for (int k = k0; k < k1; ++k) {
        const int64_t o = (int64_t)k * plane + col;
        const Uv<T> a_n = k + 1 <= nz - 2 ? c.uv(k + 1) : zero_uv;
        const Ws<T> b_n = c.ws(k + 1);
        T uvk[4] = {T(0), T(0), T(0), T(0)};
        if (k <= nz - 2) node_uv(p, c, k, o, a_k, b_k, b_n, uvk);
        T wn[2] = {T(0), T(0)};
        if (k + 1 <= nz - 1) node_w(p, k + 1, o + plane, a_k, a_n, b_n, wn);
        sxx[ty][tx] = uvk[0];
        syy[ty][tx] = uvk[1];
        sxy[ty][tx] = uvk[3];
        sxz[ty][tx] = wk[0];
        syz[ty][tx] = wk[1];
        __syncthreads();
        if (out_col) {
            const bool top = k == nz - 1;
            const T fxv = -((sxx[ty][tx + 1] - sxx[ty][tx - 1]) * p.s.cx + (sxy[ty + 1][tx] - sxy[ty - 1][tx]) * p.s.cy +
                            (wn[0] - wk[0]) * p.cz);
            const T fyv = -((sxy[ty][tx + 1] - sxy[ty][tx - 1]) * p.s.cx + (syy[ty + 1][tx] - syy[ty - 1][tx]) * p.s.cy +
                            (wn[1] - wk[1]) * p.cz);
            const T fzv = -((sxz[ty][tx + 1] - sxz[ty][tx - 1]) * p.s.cx + (syz[ty + 1][tx] - syz[ty - 1][tx]) * p.s.cy +
                            (uvk[2] - zz_m) * p.cz);
            p.fx[o] = top ? T(0) : fxv;
            p.fy[o] = top ? T(0) : fyv;
            p.fz[o] = (top || k == 0) ? T(0) : fzv;
        }
        __syncthreads();
        a_k = a_n;
        b_k = b_n;
        wk[0] = wn[0];
        wk[1] = wn[1];
        zz_m = uvk[2];
    }
}

template <typename T, typename V>
int launch_sgs_force(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv,
                     const void *wt_w, const void *const tau[6], void *fx, void *fy, void *fz, double cs,
                     cudaStream_t stream)
{
    FuseParams<T, V> p;
    p.s.u = (const V *)u; p.s.v = (const V *)v; p.s.w = (const V *)w;
    p.s.wt_uv = (const T *)wt_uv; p.s.wt_w = (const T *)wt_w;
    p.s.txx = (T *)tau[0]; p.s.txy = (T *)tau[1]; p.s.tyy = (T *)tau[2];
    p.s.tzz = (T *)tau[3]; p.s.txz = (T *)tau[4]; p.s.tyz = (T *)tau[5];
    p.s.nx = h->nx; p.s.ny = h->ny; p.s.nz = h->nz;
    p.s.cx = (T)(1.0 / (2.0 * h->dx));
    p.s.cy = (T)(1.0 / (2.0 * h->dy));
    p.s.rdz = (T)(1.0 / h->dz);
    const double lam0 = cs * cbrt(h->dx * h->dy * h->dz);
    p.s.inv_lam0_sq = (T)(1.0 / (lam0 * lam0));
    p.fx = (T *)fx; p.fy = (T *)fy; p.fz = (T *)fz;
    p.cz = (T)(1.0 / h->dz);
    dim3 block(kFuseX, kFuseY, 1);
    dim3 grid((h->nx + kFuseX - 3) / (kFuseX - 2), (h->ny + kFuseY - 3) / (kFuseY - 2),
              (h->nz + kFuseLevels - 1) / kFuseLevels);
    if (grid.y > 65535 || grid.z > 65535) return set_error(h, WMIBM_EINVAL, "grid too large for the fused launch");
    k_sgs_force<T, V><<<grid, block, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_sgs_force launch");
}

// ---------------------------------------------------------------------------
// The same march with two x-neighbouring columns per thread (FP32, nx even,
// every array aligned to two elements): the pair's centre values and its
// y-neighbours arrive as one two-element load, and the centre of each column is
// the other's x-neighbour, so a level takes 15 loads for two columns instead of
// 30, and the wall terms and the stresses move in pairs where both nodes are
// fluid.  No software pipelining here: the registers it needs would cost the
// fourth block per SM, which is worth more (measured).
template <typename T, typename V>
__device__ __forceinline__ void load2(const V *p, int64_t q, T &a, T &b)
{
    if constexpr (sizeof(V) == 8) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p + q));
        a = (T)t.x;
        b = (T)t.y;
    } else if constexpr (sizeof(V) == 4) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p + q));
        a = (T)t.x;
        b = (T)t.y;
    } else {
        const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p + q));
        a = (T)t.x;
        b = (T)t.y;
    }
}

template <typename T>
__device__ __forceinline__ void store2(T *p, int64_t q, T a, T b)
{
    if constexpr (sizeof(T) == 8)
        *reinterpret_cast<double2 *>(p + q) = make_double2(a, b);
    else
        *reinterpret_cast<float2 *>(p + q) = make_float2(a, b);
}

// Raw values of level L for the column pair (i0, i0 + 1): centres, the x-neighbours
// outside the pair (left of i0, right of i0 + 1), the y-neighbour pairs, and w above.
template <typename T>
struct Raw2 {
    T uc[2], vc[2], wup[2];
    T u_l, u_r, v_l, v_r, w_l, w_r;
    T u_jp[2], u_jm[2], v_jp[2], v_jm[2], w_jp[2], w_jm[2];
};

template <typename T, typename V>
struct Pair {
    const V *u, *v, *w;
    int64_t plane;
    int32_t nx, nz;
    int i0, il, ir, j, jm, jp;

    __device__ __forceinline__ Raw2<T> load(int L) const
    {
        Raw2<T> r;
        if (L <= nz - 2) {
            const int64_t base = (int64_t)L * plane;
            const int64_t row = base + (int64_t)j * nx, rp = base + (int64_t)jp * nx, rm = base + (int64_t)jm * nx;
            load2<T, V>(u, row + i0, r.uc[0], r.uc[1]);
            r.u_l = load_vel<V, T>(u, row + il);
            r.u_r = load_vel<V, T>(u, row + ir);
            load2<T, V>(u, rp + i0, r.u_jp[0], r.u_jp[1]);
            load2<T, V>(u, rm + i0, r.u_jm[0], r.u_jm[1]);
            load2<T, V>(v, row + i0, r.vc[0], r.vc[1]);
            r.v_l = load_vel<V, T>(v, row + il);
            r.v_r = load_vel<V, T>(v, row + ir);
            load2<T, V>(v, rp + i0, r.v_jp[0], r.v_jp[1]);
            load2<T, V>(v, rm + i0, r.v_jm[0], r.v_jm[1]);
            load2<T, V>(w, row + plane + i0, r.wup[0], r.wup[1]);
            r.w_l = load_vel<V, T>(w, row + il);
            r.w_r = load_vel<V, T>(w, row + ir);
            load2<T, V>(w, rp + i0, r.w_jp[0], r.w_jp[1]);
            load2<T, V>(w, rm + i0, r.w_jm[0], r.w_jm[1]);
        } else {
            r = Raw2<T>{};
        }
        return r;
    }
};

template <typename T, typename V>
__global__ void __launch_bounds__(256, 4) k_sgs2(SgsParams<T, V> p, int kc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i0 = 2 * t;
    if (i0 >= p.nx || j >= p.ny) return;
    const int k0 = blockIdx.z * kc;
    const int k1 = min(k0 + kc, p.nz);
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int il = i0 == 0 ? p.nx - 1 : i0 - 1, ir = i0 + 2 == p.nx ? 0 : i0 + 2;
    const int jm = j == 0 ? p.ny - 1 : j - 1, jp = j + 1 == p.ny ? 0 : j + 1;
    const Pair<T, V> P{p.u, p.v, p.w, plane, p.nx, p.nz, i0, il, ir, j, jm, jp};
    // the two columns' set-up levels, formed as the one-column march does
    Column<T, V> c[2];
    for (int q = 0; q < 2; ++q) {
        c[q].U = Field<T, V>{p.u, p.nx, p.ny, plane};
        c[q].Vf = Field<T, V>{p.v, p.nx, p.ny, plane};
        c[q].W = Field<T, V>{p.w, p.nx, p.ny, plane};
        c[q].i = i0 + q;
        c[q].j = j;
        c[q].im = q == 0 ? il : i0;
        c[q].ip = q == 0 ? i0 + 1 : ir;
        c[q].jm = jm;
        c[q].jp = jp;
        c[q].nz = p.nz; c[q].cx = p.cx; c[q].cy = p.cy; c[q].rdz = p.rdz;
    }
    Uv<T> a_prev[2], a_cur[2];
    Ws<T> b_cur[2];
    T u_c[2], v_c[2], w_c[2];
    for (int q = 0; q < 2; ++q) {
        a_prev[q] = k0 >= 1 ? c[q].uv(k0 - 1) : Uv<T>{0, 0, 0, 0};
        a_cur[q] = k0 <= p.nz - 2 ? c[q].uv(k0) : Uv<T>{0, 0, 0, 0};
        b_cur[q] = c[q].ws(k0);
        u_c[q] = k0 <= p.nz - 2 ? c[q].U.at(i0 + q, j, k0) : T(0);
        v_c[q] = k0 <= p.nz - 2 ? c[q].Vf.at(i0 + q, j, k0) : T(0);
        w_c[q] = k0 <= p.nz - 2 ? c[q].W.at(i0 + q, j, k0 + 1) : T(0);
    }
    int64_t o = (int64_t)k0 * plane + (int64_t)j * p.nx + i0;
    for (int k = k0; k < k1; ++k, o += plane) {
        const Raw2<T> raw = P.load(k + 1);
        T wt_uv[2] = {T(-1), T(-1)}, wt_w[2] = {T(-1), T(-1)};
        if (k <= p.nz - 2) load2<T, T>(p.wt_uv, o, wt_uv[0], wt_uv[1]);
        if (k >= 1) load2<T, T>(p.wt_w, o, wt_w[0], wt_w[1]);
        const int L = k + 1;
        Uv<T> a_next[2] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        Ws<T> b_next[2] = {{0, 0}, {0, 0}};
        if (L <= p.nz - 2) {
            for (int q = 0; q < 2; ++q) {
                const T u_ip = q == 0 ? raw.uc[1] : raw.u_r, u_im = q == 0 ? raw.u_l : raw.uc[0];
                const T v_ip = q == 0 ? raw.vc[1] : raw.v_r, v_im = q == 0 ? raw.v_l : raw.vc[0];
                const T w_ip = q == 0 ? w_c[1] : raw.w_r, w_im = q == 0 ? raw.w_l : w_c[0];
                a_next[q].s11 = (u_ip - u_im) * p.cx;
                a_next[q].s22 = (raw.v_jp[q] - raw.v_jm[q]) * p.cy;
                a_next[q].s12 = T(0.5) * ((raw.u_jp[q] - raw.u_jm[q]) * p.cy + (v_ip - v_im) * p.cx);
                a_next[q].s33 = (raw.wup[q] - w_c[q]) * p.rdz;
                b_next[q].s13 = T(0.5) * ((raw.uc[q] - u_c[q]) * p.rdz + (w_ip - w_im) * p.cx);
                b_next[q].s23 = T(0.5) * ((raw.vc[q] - v_c[q]) * p.rdz + (raw.w_jp[q] - raw.w_jm[q]) * p.cy);
            }
        }
        T tu[2][4], tw[2][2];
        for (int q = 0; q < 2; ++q) {
            if (wt_uv[q] >= T(0)) uv_stress(a_cur[q], b_cur[q], b_next[q], wt_uv[q], p.inv_lam0_sq, tu[q]);
            tw[q][0] = tw[q][1] = T(0);                             // the lid: no stress (Eq. 10)
            if (wt_w[q] >= T(0) && k < p.nz - 1) w_stress(a_prev[q], a_cur[q], b_cur[q], wt_w[q], p.inv_lam0_sq, tw[q]);
        }
        if (wt_uv[0] >= T(0) && wt_uv[1] >= T(0)) {                 // uv-nodes (i0, j, k), (i0 + 1, j, k)
            store2(p.txx, o, tu[0][0], tu[1][0]);
            store2(p.tyy, o, tu[0][1], tu[1][1]);
            store2(p.tzz, o, tu[0][2], tu[1][2]);
            store2(p.txy, o, tu[0][3], tu[1][3]);
        } else {
            for (int q = 0; q < 2; ++q)
                if (wt_uv[q] >= T(0)) {
                    p.txx[o + q] = tu[q][0];
                    p.tyy[o + q] = tu[q][1];
                    p.tzz[o + q] = tu[q][2];
                    p.txy[o + q] = tu[q][3];
                }
        }
        if (wt_w[0] >= T(0) && wt_w[1] >= T(0)) {                   // w-nodes; the floor is left
            store2(p.txz, o, tw[0][0], tw[1][0]);
            store2(p.tyz, o, tw[0][1], tw[1][1]);
        } else {
            for (int q = 0; q < 2; ++q)
                if (wt_w[q] >= T(0)) {
                    p.txz[o + q] = tw[q][0];
                    p.tyz[o + q] = tw[q][1];
                }
        }
        for (int q = 0; q < 2; ++q) {
            a_prev[q] = a_cur[q];
            a_cur[q] = a_next[q];
            b_cur[q] = b_next[q];
            u_c[q] = raw.uc[q];
            v_c[q] = raw.vc[q];
            w_c[q] = raw.wup[q];
        }
    }
}

template <typename T, typename V>
int launch_sgs(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv, const void *wt_w,
               void *const tau[6], double cs, cudaStream_t stream)
{
    SgsParams<T, V> p;
    p.u = (const V *)u; p.v = (const V *)v; p.w = (const V *)w;
    p.wt_uv = (const T *)wt_uv; p.wt_w = (const T *)wt_w;
    p.txx = (T *)tau[0]; p.txy = (T *)tau[1]; p.tyy = (T *)tau[2];
    p.tzz = (T *)tau[3]; p.txz = (T *)tau[4]; p.tyz = (T *)tau[5];
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz;
    p.cx = (T)(1.0 / (2.0 * h->dx));
    p.cy = (T)(1.0 / (2.0 * h->dy));
    p.rdz = (T)(1.0 / h->dz);
    const double lam0 = cs * cbrt(h->dx * h->dy * h->dz);
    p.inv_lam0_sq = (T)(1.0 / (lam0 * lam0));
    const int kc = 8;                       // levels per thread
    // FP32 only: in FP64 the pair kernel's registers cost more than its loads save (measured)
    if constexpr (sizeof(T) == 4) {
        const size_t es = sizeof(T), vs = sizeof(V);
        bool pairs = h->nx % 2 == 0;
        for (const void *q : {u, v, w})
            pairs = pairs && ((uintptr_t)q % (2 * vs)) == 0;
        for (const void *q : {wt_uv, wt_w, (const void *)tau[0], (const void *)tau[1], (const void *)tau[2],
                              (const void *)tau[3], (const void *)tau[4], (const void *)tau[5]})
            pairs = pairs && ((uintptr_t)q % (2 * es)) == 0;
        if (pairs) {
            const int half = h->nx / 2;
            dim3 block(32, 8, 1);
            dim3 grid((half + 31) / 32, (h->ny + 7) / 8, (h->nz + kc - 1) / kc);
            if (grid.y > 65535 || grid.z > 65535)
                return set_error(h, WMIBM_EINVAL, "grid too large for the SGS launch");
            k_sgs2<T, V><<<grid, block, 0, stream>>>(p, kc);
            return cuda_status(h, cudaGetLastError(), "k_sgs2 launch");
        }
    }
    const int bx = h->nx >= 64 ? 64 : 32;
    const int by = 256 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((h->nx + bx - 1) / bx, (h->ny + by - 1) / by, (h->nz + kc - 1) / kc);
    if (grid.y > 65535 || grid.z > 65535) return set_error(h, WMIBM_EINVAL, "grid too large for the SGS launch");
    k_sgs<T, V><<<grid, block, 0, stream>>>(p, kc);
    return cuda_status(h, cudaGetLastError(), "k_sgs launch");
}

}  // namespace

extern "C" int wmibm_sgs_wall_terms(wmibm_handle *h, const double *phi_uv, const double *phi_w, const double *z0,
                                    int32_t z0_is_field, void *wt_uv, void *wt_w, void *stream)
{
    ApiRange nvtx_range("wmibm_sgs_wall_terms");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!phi_uv || !phi_w || !z0 || !wt_uv || !wt_w) return set_error(h, WMIBM_EINVAL, "NULL argument");
    int st = check_device(h);
    if (st) return st;
    const int64_t n = h->n;
    const size_t es = elem_size(h->dtype);
    void *host = host_alloc(2 * n * es);
    if (!host) return set_error(h, WMIBM_ENOMEM, "host memory for the wall terms");
    const double pb = h->phi_b, kap = h->kappa;
    for (int g = 0; g < 2; ++g) {
        const double *phi = g == 0 ? phi_uv : phi_w;
        for (int64_t q = 0; q < n; ++q) {
            const double f = phi[q];
            const double zz = z0_is_field ? z0[q] : z0[0];
            // the node classes of init, with the same inclusive comparisons: uv-grid band
            // 0 <= phi <= 2 phi_b, solid phi < 0; w-grid band |phi| <= phi_b, solid phi < -phi_b
            const bool solid = g == 0 ? f < 0.0 : f < -pb;
            const bool fluid = g == 0 ? f > 2.0 * pb : f > pb;
            const double val = fluid ? 1.0 / ((kap * (f + zz)) * (kap * (f + zz))) : (solid ? -2.0 : -1.0);
            if (h->dtype == WMIBM_F64) ((double *)host)[g * n + q] = val;
            else ((float *)host)[g * n + q] = (float)val;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(wt_uv, host, n * es, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wt_w, (char *)host + n * es, n * es, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(host);
    return cuda_status(h, e, "wall terms upload");
}

extern "C" int wmibm_sgs_stress(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv,
                                const void *wt_w, void *const tau[6], double cs, void *stream)
{
    ApiRange nvtx_range("wmibm_sgs_stress");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w || !wt_uv || !wt_w || !tau) return set_error(h, WMIBM_EINVAL, "NULL argument");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    if (!(cs > 0.0)) return set_error(h, WMIBM_EINVAL, "the Smagorinsky coefficient must be positive");
    int st = check_device(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->dtype == WMIBM_F64) return launch_sgs<double, double>(h, u, v, w, wt_uv, wt_w, tau, cs, s);
    if (h->vel_dtype == WMIBM_BF16) return launch_sgs<float, __nv_bfloat16>(h, u, v, w, wt_uv, wt_w, tau, cs, s);
    return launch_sgs<float, float>(h, u, v, w, wt_uv, wt_w, tau, cs, s);
}

extern "C" int wmibm_sgs_force(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv,
                               const void *wt_w, const void *const tau[6], void *fx, void *fy, void *fz, double cs,
                               void *stream)
{
    ApiRange nvtx_range("wmibm_sgs_force");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!u || !v || !w || !wt_uv || !wt_w || !tau || !fx || !fy || !fz)
        return set_error(h, WMIBM_EINVAL, "NULL argument");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    if (!(cs > 0.0)) return set_error(h, WMIBM_EINVAL, "the Smagorinsky coefficient must be positive");
    int st = check_device(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->dtype == WMIBM_F64)
        return launch_sgs_force<double, double>(h, u, v, w, wt_uv, wt_w, tau, fx, fy, fz, cs, s);
    if (h->vel_dtype == WMIBM_BF16)
        return launch_sgs_force<float, __nv_bfloat16>(h, u, v, w, wt_uv, wt_w, tau, fx, fy, fz, cs, s);
    return launch_sgs_force<float, float>(h, u, v, w, wt_uv, wt_w, tau, fx, fy, fz, cs, s);
}
