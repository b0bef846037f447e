// Adjoint of one stage (wall stress of Sec. 3.3 of Liu & Stevens,
// arXiv:2006.03343, then f = -div tau of Eqs. 15-16 and Eq. 18) for the linear
// functional L = sum over nodes of (gx fx + gy fy + gz fz), with the per-cell
// roughness s = ln z0 as a parameter (C = kappa^2 / (ln phi_c - s)^2).
//
//   1. per band record: gam = dL/dtau at the node's stored components (the
//      transpose of the divergence, gathered from g around the node); with
//      r = U_r, rho = |r|, m = G n and q = r . m (G the symmetric matrix of gam),
//      L_node = -2 C rho q, so
//        dL/du_hat = P (-2 C (q r / rho + rho m)),  P = I - n n^T
//        dL/ds     = -2 rho q * 2 C / (ln phi_c - s)
//   2. per touched velocity node: dL/du = sum over the (record, corner) pairs of
//      the transpose map of (trilinear weight) * dL/du_hat, in ascending
//      (record, corner) order; per band cell: dL/ds = w-band part + uv-band part.
// No atomics: every output element is written by one thread in a fixed order,
// so the result is deterministic.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

#include "band.cuh"

using namespace wmibm;

namespace {

template <typename T>
struct AdjParams {
    const void *rec;
    int64_t nb_w, nrec;
    const T *gx, *gy, *gz;
    const void *u, *v, *w;
    const T *logz0;
    T log_phi_c, kappa, kappa2;
    int32_t nx, ny, nz;
    T hx, hy, hz;                 // 1 / (2 dx), 1 / (2 dy), 1 / dz
    T *grad;                      // [nrec][4]: dL/du_hat (3), dL/ds
    // gather
    const int32_t *keys, *offs, *ent;
    int64_t m_uv, m_w;
    const int32_t *band_w, *band_uv;   // ascending node lists of the two bands
    T *du, *dv, *dw, *ds;
    // zeroing of the gradient fields, by the blocks after the records' blocks
    int64_t n;                    // nodes per field
    int64_t record_blocks;
    int32_t vec16;                // the fields are 16-byte aligned and n * sizeof(T) is a multiple of 16
};

// Clears du, dv, dw (and ds) before the gather writes the touched nodes: zeroing
// block zb of nzb, grid-stride, 16-byte stores where the fields allow.
template <typename T>
__device__ void zero_gradients(const AdjParams<T> &p, int64_t zb, int64_t nzb)
{
    T *const outs[4] = {p.du, p.dv, p.dw, p.ds};
    const int64_t first = zb * kThreads + threadIdx.x, stride = nzb * kThreads;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        T *o = outs[f];
        if (!o) continue;
        if (p.vec16) {
            const int64_t n4 = p.n * (int64_t)sizeof(T) / 16;
            for (int64_t q = first; q < n4; q += stride) reinterpret_cast<float4 *>(o)[q] = make_float4(0, 0, 0, 0);
        } else {
            for (int64_t q = first; q < p.n; q += stride) o[q] = T(0);
        }
    }
}

// Blocks [0, record_blocks): one band record per thread.  The blocks after them
// clear the gradient fields meanwhile (the gather, next in the stream, writes the
// touched nodes after both).
template <typename T, typename VEL>
__global__ void __launch_bounds__(kThreads) k_adjoint_records(AdjParams<T> p)
{
    using Rec = typename RecOf<T>::type;
    if ((int64_t)blockIdx.x >= p.record_blocks) {
        zero_gradients(p, (int64_t)blockIdx.x - p.record_blocks, (int64_t)gridDim.x - p.record_blocks);
        return;
    }
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= p.nrec) return;
    T nxv, nyv, nzv, C, ax, ay, azu, azw;
    int4 ix;
    unpack(reinterpret_cast<const Rec *>(p.rec), t, nxv, nyv, nzv, C, ax, ay, azu, azw, ix);
    const bool is_w = t < p.nb_w;
    const int32_t nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t di = (ix.w & 1) ? 1 - nx : 1;
    const int64_t dj = (ix.w & 2) ? (int64_t)(1 - ny) * nx : nx;
    const T uc = trilinear<VEL, T>(reinterpret_cast<const VEL *>(p.u), ix.y, di, dj, plane, ax, ay, azu);
    const T vc = trilinear<VEL, T>(reinterpret_cast<const VEL *>(p.v), ix.y, di, dj, plane, ax, ay, azu);
    const T wc = trilinear<VEL, T>(reinterpret_cast<const VEL *>(p.w), ix.z, di, dj, plane, ax, ay, azw);
    T lg;
    if (p.logz0) {
        lg = p.log_phi_c - __ldg(p.logz0 + ix.x);
        C = p.kappa2 / (lg * lg);
    } else {
        lg = p.kappa / sqrt(C);             // C = kappa^2 / lg^2 with lg = ln(phi_c / z0) > 0
    }

    // node coordinates and its horizontal neighbours (periodic)
    const int64_t idx = ix.x;
    const int32_t k = (int32_t)(idx / plane);
    const int64_t rem = idx - (int64_t)k * plane;
    const int32_t j = (int32_t)(rem / nx);
    const int32_t i = (int32_t)(rem - (int64_t)j * nx);
    const int64_t row = idx - i, lev = idx - rem;
    const int64_t ip = row + (i + 1 == nx ? 0 : i + 1), im = row + (i == 0 ? nx - 1 : i - 1);
    const int64_t jp = lev + (int64_t)(j + 1 == ny ? 0 : j + 1) * nx + i;
    const int64_t jm = lev + (int64_t)(j == 0 ? ny - 1 : j - 1) * nx + i;
    const bool fx_on = k <= nz - 2;                  // f_x, f_y at uv level k (not the ghost level)
    const bool fz_on = k >= 1 && k <= nz - 2;        // f_z at w level k (not floor or lid)

    T mx, my, mz;                                     // m = G n
    if (is_w) {
        // txz at w level k enters f_x at uv levels k-1 and k, and f_z at w level k
        T gxz = p.hz * ((fx_on ? __ldg(p.gx + idx) : T(0)) - (k >= 1 ? __ldg(p.gx + idx - plane) : T(0)));
        T gyz = p.hz * ((fx_on ? __ldg(p.gy + idx) : T(0)) - (k >= 1 ? __ldg(p.gy + idx - plane) : T(0)));
        if (fz_on) {
            gxz += p.hx * (__ldg(p.gz + ip) - __ldg(p.gz + im));
            gyz += p.hy * (__ldg(p.gz + jp) - __ldg(p.gz + jm));
        }
        mx = T(0.5) * gxz * nzv;
        my = T(0.5) * gyz * nzv;
        mz = T(0.5) * (gxz * nxv + gyz * nyv);
    } else {
        T gxx = T(0), gxy = T(0), gyy = T(0);
        if (fx_on) {
            gxx = p.hx * (__ldg(p.gx + ip) - __ldg(p.gx + im));
            gxy = p.hy * (__ldg(p.gx + jp) - __ldg(p.gx + jm)) + p.hx * (__ldg(p.gy + ip) - __ldg(p.gy + im));
            gyy = p.hy * (__ldg(p.gy + jp) - __ldg(p.gy + jm));
        }
        // tzz at uv level k enters f_z at w levels k and k+1
        const T gzz = p.hz * ((k <= nz - 3 ? __ldg(p.gz + idx + plane) : T(0)) - (fz_on ? __ldg(p.gz + idx) : T(0)));
        mx = gxx * nxv + T(0.5) * gxy * nyv;
        my = T(0.5) * gxy * nxv + gyy * nyv;
        mz = gzz * nzv;
    }

    const T un = uc * nxv + vc * nyv + wc * nzv;
    const T rx = uc - un * nxv, ry = vc - un * nyv, rz = wc - un * nzv;
    const T rho = sqrt(rx * rx + ry * ry + rz * rz);
    T o0 = T(0), o1 = T(0), o2 = T(0), o3 = T(0);
    if (rho > T(0)) {
        const T q = rx * mx + ry * my + rz * mz;
        const T a = -T(2) * C;
        const T dx_ = a * (q * rx / rho + rho * mx);
        const T dy_ = a * (q * ry / rho + rho * my);
        const T dz_ = a * (q * rz / rho + rho * mz);
        const T nd = nxv * dx_ + nyv * dy_ + nzv * dz_;
        o0 = dx_ - nd * nxv;
        o1 = dy_ - nd * nyv;
        o2 = dz_ - nd * nzv;
        o3 = -T(2) * rho * q * (T(2) * C / lg);
    }
    T *g = p.grad + 4 * t;
    g[0] = o0;
    g[1] = o1;
    g[2] = o2;
    g[3] = o3;
}

// Position of node idx in an ascending list, or -1.
__device__ __forceinline__ int64_t find_node(const int32_t *list, int64_t n, int32_t idx)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(list + mid) < idx)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && __ldg(list + lo) == idx) ? lo : -1;
}

template <typename T>
__device__ __forceinline__ T corner_weight(int c, T ax, T ay, T az)
{
    const T wx = (c & 1) ? ax : T(1) - ax;
    const T wy = (c & 2) ? ay : T(1) - ay;
    const T wz = (c & 4) ? az : T(1) - az;
    return wx * wy * wz;
}

// Threads [0, m_uv): touched uv-grid nodes (du, dv); [m_uv, m_uv + m_w): touched
// w-grid nodes (dw); then one thread per band record for dL/ds (if wanted).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adjoint_gather(AdjParams<T> p)
{
    using Rec = typename RecOf<T>::type;
    const Rec *rec = reinterpret_cast<const Rec *>(p.rec);
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t m = p.m_uv + p.m_w;
    if (t < m) {
        const bool uv = t < p.m_uv;
        const int32_t node = __ldg(p.keys + t);
        T s0 = T(0), s1 = T(0);
        for (int32_t e = __ldg(p.offs + t); e < __ldg(p.offs + t + 1); ++e) {
            const int32_t code = __ldg(p.ent + e);
            const int64_t r = code >> 3;
            T nxv, nyv, nzv, C, ax, ay, azu, azw;
            int4 ix;
            unpack(rec, r, nxv, nyv, nzv, C, ax, ay, azu, azw, ix);
            const T wt = corner_weight<T>(code & 7, ax, ay, uv ? azu : azw);
            if (uv) {
                s0 += wt * p.grad[4 * r + 0];
                s1 += wt * p.grad[4 * r + 1];
            } else {
                s0 += wt * p.grad[4 * r + 2];
            }
        }
        if (uv) {
            p.du[node] = s0;
            p.dv[node] = s1;
        } else {
            p.dw[node] = s0;
        }
        return;
    }
    const int64_t r = t - m;
    if (!p.ds || r >= p.nrec) return;
    const int32_t idx = __ldg(&rec[r].ix).x;
    if (r < p.nb_w) {
        // the cell's uv-band record, if any, writes the sum
        if (find_node(p.band_uv, p.nrec - p.nb_w, idx) >= 0) return;
        p.ds[idx] = p.grad[4 * r + 3];
    } else {
        const int64_t tw = find_node(p.band_w, p.nb_w, idx);
        const T a = tw >= 0 ? p.grad[4 * tw + 3] : T(0);
        p.ds[idx] = a + p.grad[4 * r + 3];    // w-band part first, then the uv-band part
    }
}

int64_t corner_entries(const wmibm_handle *h, const std::vector<unsigned char> &raw, bool w_grid,
                       std::vector<int64_t> &pairs)
{
    const size_t rsize = h->dtype == WMIBM_F64 ? sizeof(RecF64) : sizeof(RecF32);
    const size_t ix_off = h->dtype == WMIBM_F64 ? offsetof(RecF64, ix) : offsetof(RecF32, ix);
    const int64_t nx = h->nx, ny = h->ny, plane = nx * ny;
    pairs.clear();
    pairs.reserve((size_t)h->nrec * 8);
    for (int64_t r = 0; r < h->nrec; ++r) {
        int4 ix;
        memcpy(&ix, raw.data() + (size_t)r * rsize + ix_off, sizeof(int4));
        const int64_t base = w_grid ? ix.z : ix.y;
        const int64_t di = (ix.w & 1) ? 1 - nx : 1;
        const int64_t dj = (ix.w & 2) ? (1 - ny) * nx : nx;
        for (int c = 0; c < 8; ++c) {
            const int64_t node = base + ((c & 1) ? di : 0) + ((c & 2) ? dj : 0) + ((c & 4) ? plane : 0);
            pairs.push_back((node << 32) | (r * 8 + c));
        }
    }
    std::sort(pairs.begin(), pairs.end());
    return (int64_t)pairs.size();
}

// Builds the transpose map of the trilinear gathers (once per handle).
int ensure_adjoint_map(wmibm_handle *h, cudaStream_t stream)
{
    if (h->adj_grad || h->nrec == 0) return WMIBM_OK;
    // entry codes (record * 8 + corner) and offsets (16 entries per record) stay below 2^31
    if (h->nrec >= (int64_t(1) << 27)) return set_error(h, WMIBM_EINVAL, "too many band records for the adjoint map");
    const size_t rsize = h->dtype == WMIBM_F64 ? sizeof(RecF64) : sizeof(RecF32);
    std::vector<unsigned char> raw((size_t)h->nrec * rsize);
    cudaError_t e = cudaMemcpyAsync(raw.data(), h->rec, raw.size(), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(h, e, "adjoint map: copy records");

    std::vector<int32_t> keys, offs, ent;
    int64_t m[2] = {0, 0};
    std::vector<int64_t> pairs;
    for (int grid = 0; grid < 2; ++grid) {       // 0: uv-grid corners, 1: w-grid corners
        corner_entries(h, raw, grid == 1, pairs);
        int64_t prev = -1;
        for (int64_t q : pairs) {
            const int64_t node = q >> 32;
            if (node != prev) {
                keys.push_back((int32_t)node);
                offs.push_back((int32_t)ent.size());
                ++m[grid];
                prev = node;
            }
            ent.push_back((int32_t)(q & 0xffffffff));
        }
    }
    offs.push_back((int32_t)ent.size());

    const size_t gbytes = (size_t)h->nrec * 4 * elem_size(h->dtype);
    e = dev_alloc(&h->adj_keys, keys.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = dev_alloc(&h->adj_offs, offs.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = dev_alloc(&h->adj_ent, ent.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = dev_alloc(&h->adj_grad, gbytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->adj_keys, keys.data(), keys.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->adj_offs, offs.data(), offs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->adj_ent, ent.data(), ent.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFree(h->adj_keys);
        cudaFree(h->adj_offs);
        cudaFree(h->adj_ent);
        cudaFree(h->adj_grad);
        h->adj_keys = h->adj_offs = h->adj_ent = nullptr;
        h->adj_grad = nullptr;
        return cuda_status(h, e, "adjoint map: upload");
    }
    h->adj_m[0] = m[0];
    h->adj_m[1] = m[1];
    return WMIBM_OK;
}

template <typename T, typename VEL>
int backward_impl(wmibm_handle *h, const void *const g[3], const void *const uvw[3], void *du, void *dv, void *dw,
                  void *dlogz0, cudaStream_t stream)
{
    AdjParams<T> p = {};
    p.rec = h->rec;
    p.nb_w = h->lists.n[WMIBM_LIST_BAND_W];
    p.nrec = h->nrec;
    p.gx = (const T *)g[0];
    p.gy = (const T *)g[1];
    p.gz = (const T *)g[2];
    p.u = uvw[0];
    p.v = uvw[1];
    p.w = uvw[2];
    p.logz0 = (const T *)h->logz0;
    p.log_phi_c = (T)log(h->phi_c);
    p.kappa = (T)h->kappa;
    p.kappa2 = (T)(h->kappa * h->kappa);
    p.nx = h->nx;
    p.ny = h->ny;
    p.nz = h->nz;
    p.hx = (T)(1.0 / (2.0 * h->dx));
    p.hy = (T)(1.0 / (2.0 * h->dy));
    p.hz = (T)(1.0 / h->dz);
    p.grad = (T *)h->adj_grad;
    p.keys = h->adj_keys;
    p.offs = h->adj_offs;
    p.ent = h->adj_ent;
    p.m_uv = h->adj_m[0];
    p.m_w = h->adj_m[1];
    p.band_w = h->lists.p[WMIBM_LIST_BAND_W];
    p.band_uv = h->lists.p[WMIBM_LIST_BAND_UV];
    p.du = (T *)du;
    p.dv = (T *)dv;
    p.dw = (T *)dw;
    p.ds = (T *)dlogz0;
    p.n = h->n;
    bool al = (h->n * (int64_t)sizeof(T)) % 16 == 0;
    const void *const outs[4] = {du, dv, dw, dlogz0};
    for (int f = 0; f < 4; ++f) al = al && ((uintptr_t)outs[f] & 15u) == 0;
    p.vec16 = al ? 1 : 0;
    // records' blocks, then zeroing blocks: about two per SM, at most one per 1024 vectors
    const int64_t b1 = (h->nrec + kThreads - 1) / kThreads;
    int64_t bz = (h->n * (int64_t)sizeof(T) / 16 + 4 * kThreads - 1) / (4 * kThreads);
    if (bz > 2 * (int64_t)h->sm_count) bz = 2 * (int64_t)h->sm_count;
    if (bz < 1) bz = 1;
    p.record_blocks = b1;
    k_adjoint_records<T, VEL><<<(unsigned)(b1 + bz), kThreads, 0, stream>>>(p);
    int st = cuda_status(h, cudaGetLastError(), "k_adjoint_records launch");
    if (st) return st;
    if (h->nrec == 0) return WMIBM_OK;
    const int64_t total = p.m_uv + p.m_w + (dlogz0 ? h->nrec : 0);
    const unsigned b2 = (unsigned)((total + kThreads - 1) / kThreads);
    k_adjoint_gather<T><<<b2, kThreads, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_adjoint_gather launch");
}

}  // namespace

extern "C" int wmibm_set_log_z0(wmibm_handle *h, const void *logz0, void *stream)
{
    ApiRange nvtx_range("wmibm_set_log_z0");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    int st = check_device(h);
    if (st) return st;
    if (logz0 && ((uintptr_t)logz0 % elem_size(h->dtype)) != 0)
        return set_error(h, WMIBM_EINVAL, "logz0 is not aligned to its element size");
    st = ensure_adjoint_map(h, (cudaStream_t)stream);
    if (st) return st;
    h->logz0 = logz0;
    return WMIBM_OK;
}

extern "C" int wmibm_backward(wmibm_handle *h, const void *const g[3], const void *const uvw[3], void *du,
                              void *dv, void *dw, void *dlogz0, void *stream)
{
    ApiRange nvtx_range("wmibm_backward");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!g || !g[0] || !g[1] || !g[2]) return set_error(h, WMIBM_EINVAL, "NULL forcing weight g");
    if (!uvw || !uvw[0] || !uvw[1] || !uvw[2]) return set_error(h, WMIBM_EINVAL, "NULL velocity pointer");
    if (!du || !dv || !dw) return set_error(h, WMIBM_EINVAL, "NULL velocity gradient pointer");
    int st = check_device(h);
    if (st) return st;
    st = ensure_adjoint_map(h, (cudaStream_t)stream);
    if (st) return st;
    if (h->dtype == WMIBM_F64) return backward_impl<double, double>(h, g, uvw, du, dv, dw, dlogz0, (cudaStream_t)stream);
    if (h->vel_dtype == WMIBM_BF16)
        return backward_impl<float, __nv_bfloat16>(h, g, uvw, du, dv, dw, dlogz0, (cudaStream_t)stream);
    return backward_impl<float, float>(h, g, uvw, du, dv, dw, dlogz0, (cudaStream_t)stream);
}
