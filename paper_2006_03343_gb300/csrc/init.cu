// One-time set-up of a terrain (Sec. 3.1 and Sec. 3.3 of Liu & Stevens,
// arXiv:2006.03343): node classes, ascending index lists, unit normals and the
// per-band-node interpolation records, all computed on the GPU in FP64.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

using namespace wmibm;

namespace {

char g_init_error[512] = "";

constexpr int kChunkItems = 8;                     // nodes per thread in the list kernels
constexpr int kChunk = kThreads * kChunkItems;     // nodes per block

// ------------------------------------------------------------------------- //
// Sec. 3.3: the six predicates, in the order of WMIBM_LIST_*.
// ------------------------------------------------------------------------- //
__device__ __forceinline__ void predicates(double pw, double puv, double pb, bool q[6])
{
    // (callers test the owned x-range first)
    q[0] = (pw >= -pb) && (pw <= pb);            // w band:  -phi_b <= phi <= phi_b
    q[1] = (puv >= 0.0) && (puv <= 2.0 * pb);    // uv band: 0 <= phi <= 2 phi_b
    q[2] = pw < -pb;                             // w solid
    q[3] = puv < 0.0;                            // uv solid
    q[4] = pw <= 0.0;                            // w body (Eq. 27)
    q[5] = puv <= 0.0;                           // uv body (Eq. 27)
}

// Whether node p lies in the owned x-range [x0, x1) (x1 == 0: every node is owned).
__device__ __forceinline__ bool owned(int64_t p, int32_t nx, int32_t x0, int32_t x1)
{
    if (x1 == 0) return true;
    const int32_t i = (int32_t)(p % nx);
    return i >= x0 && i < x1;
}

__global__ void __launch_bounds__(kThreads) k_count(const double *__restrict__ phi_uv,
                                                    const double *__restrict__ phi_w, int64_t n, double pb,
                                                    int32_t *__restrict__ counts, int64_t nblk, int32_t nx,
                                                    int32_t x0, int32_t x1)
{
    __shared__ int warp_tot[6][kThreads / 32];
    int c[6] = {0, 0, 0, 0, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int it = 0; it < kChunkItems; ++it) {
        int64_t p = base + (int64_t)it * kThreads + threadIdx.x;
        if (p < n && owned(p, nx, x0, x1)) {
            bool q[6];
            predicates(phi_w[p], phi_uv[p], pb, q);
            for (int l = 0; l < 6; ++l) c[l] += q[l] ? 1 : 0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = 0; l < 6; ++l) {
        int v = c[l];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) warp_tot[l][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += warp_tot[threadIdx.x][w];
        counts[threadIdx.x * nblk + blockIdx.x] = s;
    }
}

// Stable compaction: block b writes its matches in ascending node order starting
// at offsets[l * nblk + b] (exclusive scan of k_count's totals).
__global__ void __launch_bounds__(kThreads) k_compact(const double *__restrict__ phi_uv,
                                                      const double *__restrict__ phi_w, int64_t n, double pb,
                                                      const int64_t *__restrict__ offsets, int64_t nblk,
                                                      Lists lists, int32_t nx, int32_t x0, int32_t x1)
{
    __shared__ int warp_tot[6][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t run[6];
    for (int l = 0; l < 6; ++l) run[l] = offsets[l * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int it = 0; it < kChunkItems; ++it) {
        int64_t p = base + (int64_t)it * kThreads + threadIdx.x;
        bool q[6] = {false, false, false, false, false, false};
        if (p < n && owned(p, nx, x0, x1)) predicates(phi_w[p], phi_uv[p], pb, q);
        unsigned bal[6];
        for (int l = 0; l < 6; ++l) {
            bal[l] = __ballot_sync(0xffffffffu, q[l]);
            if (lane == 0) warp_tot[l][warp] = __popc(bal[l]);
        }
        __syncthreads();
        for (int l = 0; l < 6; ++l) {
            int before = 0, total = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                int t = warp_tot[l][w];
                before += (w < warp) ? t : 0;
                total += t;
            }
            if (q[l]) lists.p[l][run[l] + before + __popc(bal[l] & lt_mask)] = (int32_t)p;
            run[l] += total;
        }
        __syncthreads();
    }
}

struct RecParams {
    const double *phi_uv, *phi_w, *z0;
    int z0_is_field;
    const int32_t *band_w, *band_uv;
    int64_t nb_w, nb_uv;
    int32_t nx, ny, nz;
    double dx, dy, dz, phi_c, kappa;
    void *rec;
    int f64;
    unsigned long long *nclamp;   // [2]: band nodes (w, uv) whose sample point's level is clamped
};

__device__ __forceinline__ int32_t wrapi(int64_t i, int32_t n)
{
    int64_t r = i % n;
    return (int32_t)(r < 0 ? r + n : r);
}

// Per band node: n = grad(phi)/|grad(phi)| (Sec. 3.1, central differences,
// one-sided at the first and last level, (0,0,1) where the gradient vanishes),
// x_c = x + (phi_c - phi) n (Sec. 3.3), its trilinear stencil on both grids
// (periodic in x, y; z clamped to the physical levels) and C = kappa^2/ln^2(phi_c/z0).
__global__ void __launch_bounds__(kThreads) k_records(RecParams p)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nb_w + p.nb_uv) return;
    const bool is_w = t < p.nb_w;
    const int32_t idx = is_w ? p.band_w[t] : p.band_uv[t - p.nb_w];
    const double *phi = is_w ? p.phi_w : p.phi_uv;
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int32_t k = (int32_t)(idx / plane);
    const int32_t j = (int32_t)((idx - (int64_t)k * plane) / p.nx);
    const int32_t i = (int32_t)(idx - (int64_t)k * plane - (int64_t)j * p.nx);

    auto at = [&](int32_t ii, int32_t jj, int32_t kk) { return phi[((int64_t)kk * p.ny + jj) * p.nx + ii]; };
    double gx = (at(wrapi(i + 1, p.nx), j, k) - at(wrapi(i - 1, p.nx), j, k)) / (2.0 * p.dx);
    double gy = (at(i, wrapi(j + 1, p.ny), k) - at(i, wrapi(j - 1, p.ny), k)) / (2.0 * p.dy);
    double gz;
    if (k == 0)
        gz = (at(i, j, 1) - at(i, j, 0)) / p.dz;
    else if (k == p.nz - 1)
        gz = (at(i, j, k) - at(i, j, k - 1)) / p.dz;
    else
        gz = (at(i, j, k + 1) - at(i, j, k - 1)) / (2.0 * p.dz);
    double mag = sqrt(gx * gx + gy * gy + gz * gz);
    double nx, ny, nz;
    if (mag <= 1e-12) {
        nx = 0.0; ny = 0.0; nz = 1.0;
    } else {
        nx = gx / mag; ny = gy / mag; nz = gz / mag;
    }

    const double d = p.phi_c - phi[idx];
    const double xc = (double)i * p.dx + d * nx;
    const double yc = (double)j * p.dy + d * ny;
    const double zc = (is_w ? (double)k : (double)k + 0.5) * p.dz + d * nz;

    const double xi = xc / p.dx, eta = yc / p.dy;
    const double fi = floor(xi), fj = floor(eta);
    const double ax = xi - fi, ay = eta - fj;
    const int32_t i0 = wrapi((int64_t)fi, p.nx), j0 = wrapi((int64_t)fj, p.ny);

    double az[2];
    int32_t kb[2];
    bool clamped = false;
    for (int g = 0; g < 2; ++g) {          // g = 0: uv-grid, g = 1: w-grid
        double zeta = (g == 1) ? zc / p.dz : zc / p.dz - 0.5;
        const int32_t top = (g == 1) ? p.nz - 1 : p.nz - 2;
        if (zeta < 0.0 || zeta > (double)top) clamped = true;
        zeta = fmin(fmax(zeta, 0.0), (double)top);
        int32_t k0 = (int32_t)floor(zeta);
        if (k0 > top - 1) k0 = top - 1;
        kb[g] = k0;
        az[g] = zeta - (double)k0;
    }

    if (clamped) atomicAdd(p.nclamp + (is_w ? 0 : 1), 1ull);
    const double z0 = p.z0_is_field ? p.z0[idx] : p.z0[0];
    const double lg = log(p.phi_c / z0);
    const double C = (p.kappa * p.kappa) / (lg * lg);

    int4 ix;
    ix.x = idx;
    ix.y = (int32_t)(((int64_t)kb[0] * p.ny + j0) * p.nx + i0);
    ix.z = (int32_t)(((int64_t)kb[1] * p.ny + j0) * p.nx + i0);
    ix.w = (i0 == p.nx - 1 ? 1 : 0) | (j0 == p.ny - 1 ? 2 : 0);
    if (p.f64) {
        RecF64 r;
        r.n01 = make_double2(nx, ny);
        r.n2C = make_double2(nz, C);
        r.fxy = make_double2(ax, ay);
        r.fz = make_double2(az[0], az[1]);
        r.ix = ix;
        reinterpret_cast<RecF64 *>(p.rec)[t] = r;
    } else {
        RecF32 r;
        r.nC = make_float4((float)nx, (float)ny, (float)nz, (float)C);
        r.frac = make_float4((float)ax, (float)ay, (float)az[0], (float)az[1]);
        r.ix = ix;
        reinterpret_cast<RecF32 *>(p.rec)[t] = r;
    }
}

// Marks every velocity element a band stencil reads (for the algorithmic byte count).
__global__ void __launch_bounds__(kThreads) k_mark(const void *rec, int f64, int64_t nrec, int32_t nx, int32_t ny,
                                                    uint8_t *mark_uv, uint8_t *mark_w)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrec) return;
    int4 ix = f64 ? reinterpret_cast<const RecF64 *>(rec)[t].ix : reinterpret_cast<const RecF32 *>(rec)[t].ix;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t di = (ix.w & 1) ? 1 - nx : 1;
    const int64_t dj = (ix.w & 2) ? (int64_t)(1 - ny) * nx : nx;
    for (int c = 0; c < 8; ++c) {
        int64_t off = ((c & 1) ? di : 0) + ((c & 2) ? dj : 0) + ((c & 4) ? plane : 0);
        mark_uv[ix.y + off] = 1;
        mark_w[ix.z + off] = 1;
    }
}

// Marks the nodes of an ascending node list.
__global__ void __launch_bounds__(kThreads) k_mark_list(const int32_t *list, int64_t count, uint8_t *mask)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) mask[list[t]] = 1;
}

// 32-byte sectors of a field of n elements, `per` elements each (the field
// starting on a sector boundary): *out += sectors holding a marked element.
__global__ void __launch_bounds__(kThreads) k_count_sectors(const uint8_t *mask, int64_t n, int per,
                                                             unsigned long long *out)
{
    unsigned long long touched = 0;
    const int64_t nsec = (n + per - 1) / per;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsec;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = s * per, b = a + per < n ? a + per : n;
        int any = 0;
        for (int64_t e = a; e < b; ++e) any |= mask[e];
        touched += any;
    }
    for (int o = 16; o > 0; o >>= 1) touched += __shfl_down_sync(0xffffffffu, touched, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, touched);
}

__global__ void __launch_bounds__(kThreads) k_count_marks(const uint8_t *a, const uint8_t *b, int64_t n,
                                                           unsigned long long *out)
{
    unsigned long long ca = 0, cb = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        ca += a[p];
        cb += b[p];
    }
    for (int o = 16; o > 0; o >>= 1) {
        ca += __shfl_down_sync(0xffffffffu, ca, o);
        cb += __shfl_down_sync(0xffffffffu, cb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, ca);
        atomicAdd(out + 1, cb);
    }
}

// A solid node starts a run (maximal set of consecutive nodes of one x-row) if
// it is the first of the list, does not follow its predecessor, or begins a row.
__device__ __forceinline__ bool run_start(const int32_t *list, int64_t t, int32_t nx)
{
    return t == 0 || list[t] != list[t - 1] + 1 || list[t] % nx == 0;
}

__global__ void __launch_bounds__(kThreads) k_runs_count(const int32_t *list, int64_t n, int32_t nx,
                                                          int32_t *counts)
{
    __shared__ int warp_tot[kThreads / 32];
    int c = 0;
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int it = 0; it < kChunkItems; ++it) {
        const int64_t t = base + (int64_t)it * kThreads + threadIdx.x;
        if (t < n && run_start(list, t, nx)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int sacc = 0;
        for (int w = 0; w < kThreads / 32; ++w) sacc += warp_tot[w];
        counts[blockIdx.x] = sacc;
    }
}

// Writes the runs (first node index, length) in ascending order.
__global__ void __launch_bounds__(kThreads) k_runs_write(const int32_t *list, int64_t n, int32_t nx,
                                                          const int64_t *offsets, int2 *runs)
{
    __shared__ int warp_tot[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t run = offsets[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int it = 0; it < kChunkItems; ++it) {
        const int64_t t = base + (int64_t)it * kThreads + threadIdx.x;
        const bool q = t < n && run_start(list, t, nx);
        const unsigned bal = __ballot_sync(0xffffffffu, q);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            before += (w < warp) ? warp_tot[w] : 0;
            total += warp_tot[w];
        }
        if (q) {
            int32_t len = 1;
            while (t + len < n && list[t + len] == list[t] + len && (list[t] + len) % nx != 0) ++len;
            runs[run + before + __popc(bal & ((1u << lane) - 1u))] = make_int2(list[t], len);
        }
        run += total;
        __syncthreads();
    }
}

void free_handle(wmibm_handle *h)
{
    for (int g = 0; h && g < 2; ++g)
        if (h->runs[g]) cudaFree(h->runs[g]);
    if (!h) return;
    if (h->dev_status) cudaFree(h->dev_status);
    for (int l = 0; l < 6; ++l)
        if (h->lists.p[l]) cudaFree(h->lists.p[l]);
    if (h->rec) cudaFree(h->rec);
    if (h->partials) cudaFree(h->partials);
    if (h->ticket) cudaFree(h->ticket);
    if (h->sacc) cudaFree(h->sacc);
    if (h->adj_keys) cudaFree(h->adj_keys);
    if (h->adj_offs) cudaFree(h->adj_offs);
    if (h->adj_ent) cudaFree(h->adj_ent);
    if (h->adj_grad) cudaFree(h->adj_grad);
    spectral_free(h);
    free(h);
}

}  // namespace

namespace wmibm {

int set_error(wmibm_handle *h, int status, const char *fmt, ...)
{
    char *buf = h ? h->err : g_init_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return status;
}

int cuda_status(wmibm_handle *h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return WMIBM_OK;
    return set_error(h, e == cudaErrorMemoryAllocation ? WMIBM_ENOMEM : WMIBM_ECUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

int check_device(wmibm_handle *h)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(h, e, "cudaGetDevice");
    if (dev != h->device)
        return set_error(h, WMIBM_ESTATE, "current device %d is not the handle's device %d", dev, h->device);
    return WMIBM_OK;
}

}  // namespace wmibm

#define TRY(expr, what)                                            \
    do {                                                           \
        int _st = cuda_status(nullptr, (expr), what);              \
        if (_st != WMIBM_OK) {                                     \
            status = _st;                                          \
            goto fail;                                             \
        }                                                          \
    } while (0)

extern "C" int wmibm_init(wmibm_handle **out, const wmibm_grid *g, const double *phi_uv, const double *phi_w,
                          const double *z0, int32_t z0_is_field, double phi_c, const wmibm_opts *opts,
                          void *stream_)
{
    ApiRange nvtx_range("wmibm_init");
    cudaStream_t stream = (cudaStream_t)stream_;
    g_init_error[0] = 0;
    fault_arm();
    if (!out) return set_error(nullptr, WMIBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g || !phi_uv || !phi_w || !z0) return set_error(nullptr, WMIBM_EINVAL, "NULL grid, phi or z0");
    if (g->nx < 1 || g->ny < 1 || g->nz < 3)
        return set_error(nullptr, WMIBM_EINVAL, "grid %d x %d x %d: need nx, ny >= 1 and nz >= 3", g->nx, g->ny, g->nz);
    if (!(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0) || !isfinite(g->lx) || !isfinite(g->ly) || !isfinite(g->lz))
        return set_error(nullptr, WMIBM_EINVAL, "domain lengths must be positive and finite");
    const int64_t n = (int64_t)g->nx * g->ny * g->nz;
    if (n >= ((int64_t)1 << 31) - 16) return set_error(nullptr, WMIBM_EINVAL, "grid has %lld nodes (>= 2^31)", (long long)n);

    wmibm_opts o = {0.0, 0.0, WMIBM_F32, WMIBM_F32, WMIBM_ZCLAMP_CLAMP, 0, 0};
    if (opts) o = *opts;
    if (!(o.own_x0 == 0 && o.own_x1 == 0) && !(o.own_x0 >= 0 && o.own_x0 < o.own_x1 && o.own_x1 <= g->nx))
        return set_error(nullptr, WMIBM_EINVAL, "owned x-range [%d, %d) must lie in [0, nx = %d)", o.own_x0,
                         o.own_x1, g->nx);
    if (o.zclamp != WMIBM_ZCLAMP_CLAMP && o.zclamp != WMIBM_ZCLAMP_REJECT)
        return set_error(nullptr, WMIBM_EINVAL, "zclamp must be WMIBM_ZCLAMP_CLAMP or WMIBM_ZCLAMP_REJECT");
    const double dz = g->lz / (double)(g->nz - 1);
    if (!(o.phi_b > 0)) o.phi_b = 0.5 * dz;
    if (!(o.kappa > 0)) o.kappa = 0.4;
    if (o.dtype != WMIBM_F32 && o.dtype != WMIBM_F64) return set_error(nullptr, WMIBM_EINVAL, "dtype must be F32 or F64");
    if (!(o.vel_dtype == o.dtype || (o.dtype == WMIBM_F32 && o.vel_dtype == WMIBM_BF16)))
        return set_error(nullptr, WMIBM_EINVAL, "vel_dtype must equal dtype, or be BF16 with an F32 dtype");
    if (!isfinite(o.phi_b) || !isfinite(o.kappa)) return set_error(nullptr, WMIBM_EINVAL, "phi_b and kappa must be finite");
    if (!(phi_c >= 2.0 * o.phi_b) || !isfinite(phi_c))
        return set_error(nullptr, WMIBM_EINVAL, "phi_c = %g must be finite and >= 2 phi_b = %g", phi_c, 2.0 * o.phi_b);
    const int64_t nz0 = z0_is_field ? n : 1;
    for (int64_t p = 0; p < nz0; ++p)
        if (!(z0[p] > 0.0 && z0[p] < phi_c))
            return set_error(nullptr, WMIBM_EINVAL, "z0[%lld] = %g outside (0, phi_c = %g)", (long long)p, z0[p], phi_c);
    for (int64_t p = 0; p < n; ++p)
        if (!isfinite(phi_uv[p]) || !isfinite(phi_w[p]))
            return set_error(nullptr, WMIBM_EINVAL, "non-finite phi at node %lld", (long long)p);

    int status = WMIBM_OK;
    double *d_phi_uv = nullptr, *d_phi_w = nullptr, *d_z0 = nullptr;
    int32_t *d_counts = nullptr;
    int64_t *d_offsets = nullptr;
    uint8_t *d_mark = nullptr;
    int32_t *d_counts2 = nullptr;
    int64_t *d_offsets2 = nullptr;
    unsigned long long *d_marks = nullptr;
    const int64_t nblk = (n + kChunk - 1) / kChunk;
    std::vector<int32_t> counts(6 * nblk);
    std::vector<int64_t> offsets(6 * nblk);
    unsigned long long marks[4] = {0, 0, 0, 0};
    // 32-byte sectors: velocity sectors read (uv grid, w grid); stress sectors
    // written (w grid, uv grid)
    unsigned long long sectors[4] = {0, 0, 0, 0};

    wmibm_handle *h = (wmibm_handle *)host_alloc(sizeof(wmibm_handle));
    if (!h) return set_error(nullptr, WMIBM_ENOMEM, "host allocation failed");
    TRY(cudaGetDevice(&h->device), "cudaGetDevice");
    h->nx = g->nx; h->ny = g->ny; h->nz = g->nz;
    h->lx = g->lx; h->ly = g->ly; h->lz = g->lz;
    h->dx = g->lx / (double)g->nx;
    h->dy = g->ly / (double)g->ny;
    h->dz = dz;
    h->phi_b = o.phi_b; h->kappa = o.kappa; h->phi_c = phi_c;
    fault_wait_settings(&h->wait_ns, &h->hold_release);
    h->dtype = o.dtype; h->vel_dtype = o.vel_dtype;
    h->n = n;

    TRY(dev_alloc(&d_phi_uv, n * sizeof(double)), "cudaMalloc phi_uv");
    TRY(dev_alloc(&d_phi_w, n * sizeof(double)), "cudaMalloc phi_w");
    TRY(dev_alloc(&d_z0, nz0 * sizeof(double)), "cudaMalloc z0");
    TRY(dev_alloc(&d_counts, 6 * nblk * sizeof(int32_t)), "cudaMalloc counts");
    TRY(dev_alloc(&d_offsets, 6 * nblk * sizeof(int64_t)), "cudaMalloc offsets");
    TRY(cudaMemcpyAsync(d_phi_uv, phi_uv, n * sizeof(double), cudaMemcpyHostToDevice, stream), "copy phi_uv");
    TRY(cudaMemcpyAsync(d_phi_w, phi_w, n * sizeof(double), cudaMemcpyHostToDevice, stream), "copy phi_w");
    TRY(cudaMemcpyAsync(d_z0, z0, nz0 * sizeof(double), cudaMemcpyHostToDevice, stream), "copy z0");

    k_count<<<(unsigned)nblk, kThreads, 0, stream>>>(d_phi_uv, d_phi_w, n, o.phi_b, d_counts, nblk, g->nx, o.own_x0,
                                                     o.own_x1);
    TRY(cudaGetLastError(), "k_count launch");
    TRY(cudaMemcpyAsync(counts.data(), d_counts, 6 * nblk * sizeof(int32_t), cudaMemcpyDeviceToHost, stream),
        "copy counts");
    TRY(cudaStreamSynchronize(stream), "k_count");
    for (int l = 0; l < 6; ++l) {
        int64_t s = 0;
        for (int64_t b = 0; b < nblk; ++b) {
            offsets[l * nblk + b] = s;
            s += counts[l * nblk + b];
        }
        h->lists.n[l] = s;
        TRY(dev_alloc(&h->lists.p[l], std::max<int64_t>(s, 1) * sizeof(int32_t)), "cudaMalloc list");
    }
    TRY(cudaMemcpyAsync(d_offsets, offsets.data(), 6 * nblk * sizeof(int64_t), cudaMemcpyHostToDevice, stream),
        "copy offsets");
    k_compact<<<(unsigned)nblk, kThreads, 0, stream>>>(d_phi_uv, d_phi_w, n, o.phi_b, d_offsets, nblk, h->lists,
                                                       g->nx, o.own_x0, o.own_x1);
    TRY(cudaGetLastError(), "k_compact launch");

    h->nrec = h->lists.n[0] + h->lists.n[1];
    // [0, 1]: distinct velocity elements the band stencils read on each grid;
    // [2, 3]: band nodes (w, uv) whose sample point's level is clamped;
    // [4, 5]: velocity sectors read (uv grid, w grid); [6, 7]: stress sectors written (w grid, uv grid)
    TRY(dev_alloc(&d_marks, 8 * sizeof(unsigned long long)), "cudaMalloc mark counts");
    TRY(cudaMemsetAsync(d_marks, 0, 8 * sizeof(unsigned long long), stream), "memset mark counts");
    {
        const size_t rec_size = o.dtype == WMIBM_F64 ? sizeof(RecF64) : sizeof(RecF32);
        TRY(dev_alloc(&h->rec, std::max<int64_t>(h->nrec, 1) * rec_size), "cudaMalloc records");
        if (h->nrec > 0) {
            RecParams rp;
            rp.phi_uv = d_phi_uv; rp.phi_w = d_phi_w; rp.z0 = d_z0; rp.z0_is_field = z0_is_field ? 1 : 0;
            rp.band_w = h->lists.p[0]; rp.band_uv = h->lists.p[1];
            rp.nb_w = h->lists.n[0]; rp.nb_uv = h->lists.n[1];
            rp.nx = h->nx; rp.ny = h->ny; rp.nz = h->nz;
            rp.dx = h->dx; rp.dy = h->dy; rp.dz = h->dz; rp.phi_c = phi_c; rp.kappa = o.kappa;
            rp.rec = h->rec; rp.f64 = o.dtype == WMIBM_F64;
            rp.nclamp = d_marks + 2;
            k_records<<<(unsigned)((h->nrec + kThreads - 1) / kThreads), kThreads, 0, stream>>>(rp);
            TRY(cudaGetLastError(), "k_records launch");
        }
        TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device), "SM count");
        h->partial_blocks = std::max<int64_t>((h->nrec + kThreads - 1) / kThreads, 16 * (int64_t)h->sm_count);
        TRY(dev_alloc(&h->partials, h->partial_blocks * kStatVals * elem_size(o.dtype)), "cudaMalloc partials");
        // [0] last-block ticket of the wall kernel, [1] wall-done and [2] exit counters of
        // the fused step launch; all stay 0 between calls
        TRY(dev_alloc(&h->ticket, 8 * sizeof(unsigned int)), "cudaMalloc ticket");
        TRY(cudaMemsetAsync(h->ticket, 0, 8 * sizeof(unsigned int), stream), "memset ticket");
        TRY(dev_alloc(&h->sacc, 8 * sizeof(double)), "cudaMalloc stats accumulator");
        TRY(cudaMemsetAsync(h->sacc, 0, 8 * sizeof(double), stream), "memset stats accumulator");

        // algorithmic bytes: distinct velocity elements read by the band stencils
        TRY(dev_alloc(&d_mark, 2 * n), "cudaMalloc marks");
        TRY(cudaMemsetAsync(d_mark, 0, 2 * n, stream), "memset marks");
        if (h->nrec > 0) {
            k_mark<<<(unsigned)((h->nrec + kThreads - 1) / kThreads), kThreads, 0, stream>>>(
                h->rec, o.dtype == WMIBM_F64, h->nrec, h->nx, h->ny, d_mark, d_mark + n);
            TRY(cudaGetLastError(), "k_mark launch");
        }
        k_count_marks<<<1024, kThreads, 0, stream>>>(d_mark, d_mark + n, n, d_marks);
        TRY(cudaGetLastError(), "k_count_marks launch");
        {
            // the same reads and the stress writes at the 32-byte sector granularity of
            // the memory system: the velocity sectors the stencils touch, then the
            // stress sectors the wall stage writes (band and solid nodes of a grid)
            const int per_v = 32 / (int)elem_size(o.vel_dtype), per_e = 32 / (int)elem_size(o.dtype);
            k_count_sectors<<<1024, kThreads, 0, stream>>>(d_mark, n, per_v, d_marks + 4);
            TRY(cudaGetLastError(), "k_count_sectors launch");
            k_count_sectors<<<1024, kThreads, 0, stream>>>(d_mark + n, n, per_v, d_marks + 5);
            TRY(cudaGetLastError(), "k_count_sectors launch");
            TRY(cudaMemsetAsync(d_mark, 0, 2 * n, stream), "memset marks");   // stream order: after the counts
            // lists 0 and 2 (w band, w solid) mark the w grid, lists 1 and 3 the uv grid
            for (int l = 0; l < 4; ++l) {
                if (h->lists.n[l] == 0) continue;
                uint8_t *mask = (l == 0 || l == 2) ? d_mark + n : d_mark;
                k_mark_list<<<(unsigned)((h->lists.n[l] + kThreads - 1) / kThreads), kThreads, 0, stream>>>(
                    h->lists.p[l], h->lists.n[l], mask);
                TRY(cudaGetLastError(), "k_mark_list launch");
            }
            k_count_sectors<<<1024, kThreads, 0, stream>>>(d_mark + n, n, per_e, d_marks + 6);
            TRY(cudaGetLastError(), "k_count_sectors launch");
            k_count_sectors<<<1024, kThreads, 0, stream>>>(d_mark, n, per_e, d_marks + 7);
            TRY(cudaGetLastError(), "k_count_sectors launch");
            TRY(cudaMemcpyAsync(sectors, d_marks + 4, sizeof(sectors), cudaMemcpyDeviceToHost, stream),
                "copy sector counts");
            TRY(cudaMemcpyAsync(marks, d_marks, sizeof(marks), cudaMemcpyDeviceToHost, stream), "copy mark counts");
            TRY(cudaStreamSynchronize(stream), "init kernels");
        }
        h->nzclamp[0] = (int64_t)marks[2];
        h->nzclamp[1] = (int64_t)marks[3];
        if (o.zclamp == WMIBM_ZCLAMP_REJECT && marks[2] + marks[3] > 0) {
            status = set_error(nullptr, WMIBM_EINVAL,
                               "%llu w-band and %llu uv-band sample points lie outside the physical levels "
                               "(zclamp = REJECT)", marks[2], marks[3]);
            goto fail;
        }

        // levels holding band or solid nodes (first and last entry of each sorted
        // list): stencil stages at levels [lo - 1, hi + 1] read entries the wall
        // model writes
        {
            int32_t lo = INT32_MAX, hi = -1;
            for (int l = 0; l < 4; ++l) {
                if (h->lists.n[l] == 0) continue;
                int32_t ends[2];
                TRY(cudaMemcpyAsync(&ends[0], h->lists.p[l], sizeof(int32_t), cudaMemcpyDeviceToHost, stream),
                    "copy list head");
                TRY(cudaMemcpyAsync(&ends[1], h->lists.p[l] + h->lists.n[l] - 1, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, stream), "copy list tail");
                TRY(cudaStreamSynchronize(stream), "list ends");
                const int64_t plane = (int64_t)h->nx * h->ny;
                lo = std::min<int32_t>(lo, (int32_t)(ends[0] / plane));
                hi = std::max<int32_t>(hi, (int32_t)(ends[1] / plane));
            }
            if (hi < 0) {
                h->dirty_lo = 0;
                h->dirty_hi = 0;
            } else {
                h->dirty_lo = std::max(0, lo - 1);
                h->dirty_hi = std::min(h->nz, hi + 2);
            }
        }
        // solid runs along x (used by the fused step to zero solid stresses)
        for (int gsel = 0; gsel < 2; ++gsel) {
            const int32_t *solid = h->lists.p[gsel == 0 ? WMIBM_LIST_SOLID_W : WMIBM_LIST_SOLID_UV];
            const int64_t nsolid = h->lists.n[gsel == 0 ? WMIBM_LIST_SOLID_W : WMIBM_LIST_SOLID_UV];
            const int64_t sblk = std::max<int64_t>((nsolid + kChunk - 1) / kChunk, 1);
            std::vector<int32_t> rc(sblk, 0);
            std::vector<int64_t> ro(sblk, 0);
            TRY(dev_alloc(&d_counts2, sblk * sizeof(int32_t)), "cudaMalloc run counts");
            TRY(dev_alloc(&d_offsets2, sblk * sizeof(int64_t)), "cudaMalloc run offsets");
            TRY(cudaMemsetAsync(d_counts2, 0, sblk * sizeof(int32_t), stream), "memset run counts");
            if (nsolid > 0) {
                k_runs_count<<<(unsigned)sblk, kThreads, 0, stream>>>(solid, nsolid, h->nx, d_counts2);
                TRY(cudaGetLastError(), "k_runs_count launch");
            }
            TRY(cudaMemcpyAsync(rc.data(), d_counts2, sblk * sizeof(int32_t), cudaMemcpyDeviceToHost, stream),
                "copy run counts");
            TRY(cudaStreamSynchronize(stream), "k_runs_count");
            int64_t nr = 0;
            for (int64_t b = 0; b < sblk; ++b) {
                ro[b] = nr;
                nr += rc[b];
            }
            h->nruns[gsel] = nr;
            TRY(dev_alloc(&h->runs[gsel], std::max<int64_t>(nr, 1) * sizeof(int2)), "cudaMalloc runs");
            TRY(cudaMemcpyAsync(d_offsets2, ro.data(), sblk * sizeof(int64_t), cudaMemcpyHostToDevice, stream),
                "copy run offsets");
            if (nsolid > 0) {
                k_runs_write<<<(unsigned)sblk, kThreads, 0, stream>>>(solid, nsolid, h->nx, d_offsets2,
                                                                        h->runs[gsel]);
                TRY(cudaGetLastError(), "k_runs_write launch");
            }
            TRY(cudaStreamSynchronize(stream), "k_runs_write");
            cudaFree(d_counts2);
            cudaFree(d_offsets2);
            d_counts2 = nullptr;
            d_offsets2 = nullptr;
        }
        TRY(dev_alloc(&h->dev_status, sizeof(int)), "cudaMalloc status");
        TRY(cudaMemsetAsync(h->dev_status, 0, sizeof(int), stream), "memset status");
        TRY(cudaStreamSynchronize(stream), "init state");
        status = spectral_setup(h, stream);
        if (status != WMIBM_OK) goto fail;

        const int64_t es = (int64_t)elem_size(o.dtype), vs = (int64_t)elem_size(o.vel_dtype);
        const int64_t *L = h->lists.n;
        const int64_t nruns = h->nruns[0] + h->nruns[1];
        h->traffic[0] = h->nrec * (int64_t)rec_size + (int64_t)(2 * marks[0] + marks[1]) * vs +
                        (2 * L[0] + 4 * L[1]) * es + (int64_t)sizeof(int2) * nruns + (2 * L[2] + 4 * L[3]) * es;
        // the wall stage at sector granularity: writes (every stress sector written) ...
        h->traffic[6] = 32 * (int64_t)(2 * sectors[2] + 4 * sectors[3]);
        // ... and reads: records, velocity sectors, run descriptors, and each written
        // stress sector once (a store that does not cover its whole sector makes the
        // L2 read the sector from memory first; the stage's band stores are scattered
        // and its solid runs start anywhere, so hardly any store covers a sector whole)
        h->traffic[5] = h->nrec * (int64_t)rec_size + 32 * (int64_t)(2 * sectors[0] + sectors[1]) +
                        (int64_t)sizeof(int2) * nruns + h->traffic[6];
        h->traffic[1] = 9 * n * es;
        h->traffic[2] = 4 * (L[4] + L[5]) + (L[4] + 2 * L[5]) * vs;
        h->traffic[3] = h->traffic[2] + (L[4] + 2 * L[5]) * es;
        // fused pass: the force stream plus the wall-stress work
        h->traffic[4] = h->traffic[1] + h->traffic[0];
    }

    cudaFree(d_phi_uv);
    cudaFree(d_phi_w);
    cudaFree(d_z0);
    cudaFree(d_counts);
    cudaFree(d_offsets);
    cudaFree(d_mark);
    cudaFree(d_marks);
    *out = h;
    return WMIBM_OK;

fail:
    if (stream) cudaStreamSynchronize(stream);
    cudaFree(d_counts2);
    cudaFree(d_offsets2);
    cudaFree(d_phi_uv);
    cudaFree(d_phi_w);
    cudaFree(d_z0);
    cudaFree(d_counts);
    cudaFree(d_offsets);
    cudaFree(d_mark);
    cudaFree(d_marks);
    free_handle(h);
    return status;
}

extern "C" int64_t wmibm_list_size(const wmibm_handle *h, int32_t which)
{
    if (!h || which < 0 || which > 5) return -1;
    return h->lists.n[which];
}

extern "C" int wmibm_export_list(wmibm_handle *h, int32_t which, int32_t *dst, int64_t cap, void *stream)
{
    ApiRange nvtx_range("wmibm_export_list");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (which < 0 || which > 5) return set_error(h, WMIBM_EINVAL, "list %d does not exist", which);
    if (!dst || cap < h->lists.n[which])
        return set_error(h, WMIBM_EINVAL, "destination holds %lld entries, list has %lld", (long long)cap,
                         (long long)h->lists.n[which]);
    int st = check_device(h);
    if (st) return st;
    if (h->lists.n[which] == 0) return WMIBM_OK;
    cudaError_t e = cudaMemcpyAsync(dst, h->lists.p[which], h->lists.n[which] * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return cuda_status(h, e, "export list");
}

extern "C" int64_t wmibm_traffic_bytes(const wmibm_handle *h, int32_t which)
{
    if (!h || which < 0 || which > 6) return -1;
    return h->traffic[which];
}

extern "C" void wmibm_destroy(wmibm_handle *h)
{
    ApiRange nvtx_range("wmibm_destroy");
    if (!h) return;
    cudaDeviceSynchronize();
    free_handle(h);
}

extern "C" const char *wmibm_status_string(int status)
{
    switch (status) {
    case WMIBM_OK: return "ok";
    case WMIBM_EINVAL: return "invalid argument";
    case WMIBM_ENOMEM: return "out of memory";
    case WMIBM_ECUDA: return "CUDA error";
    case WMIBM_ESTATE: return "invalid state";
    case WMIBM_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

extern "C" const char *wmibm_last_error(const wmibm_handle *h)
{
    return h ? h->err : g_init_error;
}

extern "C" int wmibm_set_tuning(wmibm_handle *h, const wmibm_tuning *t)
{
    ApiRange nvtx_range("wmibm_set_tuning");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!t) return set_error(h, WMIBM_EINVAL, "NULL tuning");
    if (t->force_path < 0 || t->force_path > 6) return set_error(h, WMIBM_EINVAL, "force_path must be 0..6");
    if (t->wall_chunk < 0 || t->wall_chunk > 65536) return set_error(h, WMIBM_EINVAL, "wall_chunk must be 0..65536");
    if (t->dyn_chunk < 0 || t->dyn_chunk > 4096) return set_error(h, WMIBM_EINVAL, "dyn_chunk must be 0..4096");
    if (t->wall_grid < 0 || t->wall_grid > 32) return set_error(h, WMIBM_EINVAL, "wall_grid must be 0..32");
    if (!(t->rows == 0 || t->rows == 1 || t->rows == 2 || t->rows == 4))
        return set_error(h, WMIBM_EINVAL, "rows must be 0, 1, 2 or 4");
    if (t->stages != 0 && (t->stages < 2 || t->stages > 8)) return set_error(h, WMIBM_EINVAL, "stages must be 2..8");
    if (t->consumer_warps < 0 || t->consumer_warps > 12)
        return set_error(h, WMIBM_EINVAL, "consumer_warps must be 0..12");
    if (t->wall_warps < 0 || t->wall_warps > 8) return set_error(h, WMIBM_EINVAL, "wall_warps must be 0..8");
    if (t->blocks_per_sm < 0 || t->direct_bx < 0 || t->direct_by < 0 || t->direct_kc < 0)
        return set_error(h, WMIBM_EINVAL, "negative tuning field");
    if (t->direct_bx * (t->direct_by > 0 ? t->direct_by : 1) > 1024)
        return set_error(h, WMIBM_EINVAL, "direct-load block too large");
    h->tuning = *t;
    return WMIBM_OK;
}

extern "C" int wmibm_get_tuning(const wmibm_handle *h, wmibm_tuning *t)
{
    if (!h || !t) return WMIBM_EINVAL;
    *t = h->tuning;
    return WMIBM_OK;
}

extern "C" int wmibm_device_status(wmibm_handle *h, int32_t *out, void *stream)
{
    ApiRange nvtx_range("wmibm_device_status");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!out) return set_error(h, WMIBM_EINVAL, "NULL output");
    int st = check_device(h);
    if (st) return st;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->dev_status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dev_status, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(h, e, "device status");
    *out = v == 0 ? WMIBM_OK : WMIBM_ETIMEOUT;
    return WMIBM_OK;
}
