// Exact signed distance to a height field (Sec. 3.1 of Liu & Stevens,
// arXiv:2006.03343: phi = +d in the fluid, -d in the solid, d the minimum
// distance to the immersed boundary), for terrain given as heights h[j][i] at
// the column nodes.  The boundary is the piecewise-linear surface through the
// samples, each cell split along its (i, j)-(i+1, j+1) diagonal into two flat
// triangles, periodic in x and y.
//
// Each column (i, j) is shared by eight threads, each writing every 8th level of
// both grids there.  Only
// levels within `reach` of the heights around the column can be nearer than
// `reach` to the surface; every other level keeps z - h[j][i], which has the
// right sign and a magnitude above the reach.  For a level that can, the
// distance starts at |z - h[j][i]| (the vertex straight below or above is on
// the surface) and visits the window of cells within `reach` horizontally in
// ascending horizontal distance (a list built on the host and passed in the
// kernel's parameters), stopping once that distance alone exceeds the best so
// far; a cell is skipped when the horizontal gap and the vertical gap to its
// height range together exceed it.  A visited cell gives the face distance of
// each triangle whose projection lands inside it, and the distances to the
// edges not dominated by such a face.  FP64 throughout: the result feeds the
// FP64 classification of wmibm_init.
#include "internal.cuh"

#include <algorithm>
#include <vector>

using namespace wmibm;

namespace {

constexpr int kSdfCols = 32;     // columns per block: one row segment
constexpr int kSdfLanes = 8;     // warps per block, each taking every 8th level
constexpr int kSdfMaxCells = 1024;
constexpr int kSdfSmemCap = 20 * 1024;   // bytes for each of the z table and the height tiles

struct SdfParams {
    const double *h;
    double *phi_uv, *phi_w;
    int32_t nx, ny, nz, ncells;
    int32_t wx, wy, segs, tw;    // window half-widths in cells, row segments per row, tile width
    double dx, dy, dz, rdx, rdy, reach;
    float dxf, dyf, rdxf, rdyf, spanf;   // spanf: horizontal extent of the window, (wx + wy + 2) cells
    int8_t ca[kSdfMaxCells], cb[kSdfMaxCells];   // window cells (i + ca, j + cb), nearest first
};

__device__ __forceinline__ int wrap_index(int q, int n)
{
    if (q >= 0 && q < n) return q;
    q %= n;
    return q < 0 ? q + n : q;
}

// squared distance from the origin to the segment P -> Q (nearest point
// P + t (Q - P), t the projection parameter clamped to [0, 1])
template <typename T>
__device__ __forceinline__ T seg2(T px, T py, T pz, T qx, T qy, T qz)
{
    const T wx = -px, wy = -py, wz = -pz;
    const T ex = qx - px, ey = qy - py, ez = qz - pz;
    const T we = wx * ex + wy * ey + wz * ez;
    T t = T(0);
    if (we > T(0)) {
        const T ee = ex * ex + ey * ey + ez * ez;
        t = we >= ee ? T(1) : we / ee;
    }
    const T rx = wx - t * ex, ry = wy - t * ey, rz = wz - t * ez;
    return rx * rx + ry * ry + rz * rz;
}

// squared distance from the node, at the origin, to the two triangles of the
// cell whose corner A sits at (x0, y0); e00 = h(A) - z, e10 at (x0 + dx, y0),
// e01 at (x0, y0 + dy), e11 at (x0 + dx, y0 + dy): heights relative to the node
template <typename T>
__device__ T cell2(T x0, T y0, T dx, T dy, T rdx, T rdy, T e00, T e10, T e01, T e11)
{
    const T x1 = x0 + dx, y1 = y0 + dy;
    T best = T(INFINITY);
    // lower triangle A(x0,y0) B(x1,y0) C(x1,y1): plane e00 + s1x (x - x0) + s1y (y - y0);
    // c1 = the node's height above that plane
    const T s1x = (e10 - e00) * rdx, s1y = (e11 - e10) * rdy;
    const T c1 = s1x * x0 + s1y * y0 - e00;
    const T t1 = c1 / (T(1) + s1x * s1x + s1y * s1y);
    // orthogonal projection of the node, relative to A
    const T u1 = t1 * s1x - x0, v1 = t1 * s1y - y0;
    const bool in1 = u1 <= dx && v1 >= T(0) && v1 * dx <= u1 * dy;
    if (in1) best = c1 * t1;
    // upper triangle A C D(x0,y1)
    const T s2x = (e11 - e01) * rdx, s2y = (e01 - e00) * rdy;
    const T c2 = s2x * x0 + s2y * y0 - e00;
    const T t2 = c2 / (T(1) + s2x * s2x + s2y * s2y);
    const T u2 = t2 * s2x - x0, v2 = t2 * s2y - y0;
    const bool in2 = u2 >= T(0) && v2 <= dy && v2 * dx >= u2 * dy;
    if (in2) best = fmin(best, c2 * t2);
    // edges of a triangle whose face did not project inside it; the diagonal
    // belongs to both, so either face dominates it
    if (!in1) {
        best = fmin(best, seg2<T>(x0, y0, e00, x1, y0, e10));
        best = fmin(best, seg2<T>(x1, y0, e10, x1, y1, e11));
    }
    if (!in2) {
        best = fmin(best, seg2<T>(x1, y1, e11, x0, y1, e01));
        best = fmin(best, seg2<T>(x0, y1, e01, x0, y0, e00));
    }
    if (!in1 && !in2) best = fmin(best, seg2<T>(x0, y0, e00, x1, y1, e11));
    return best;
}

// Heights around one column: from the block's shared tiles (TILE) or from
// global memory.  Offsets (a, b) are relative to the column, |a| <= wx, |b| <= wy.
template <bool TILE>
struct Heights {
    const SdfParams &p;
    const double *dt;
    const float *ft;
    int c, i, j;
    __device__ double d(int a, int b) const
    {
        if (TILE) return dt[(b + p.wy) * p.tw + c + a + p.wx];
        return __ldg(p.h + (int64_t)wrap_index(j + b, p.ny) * p.nx + wrap_index(i + a, p.nx));
    }
    __device__ float f(int a, int b) const
    {
        if (TILE) return ft[(b + p.wy) * p.tw + c + a + p.wx];
        return (float)d(a, b);
    }
};

__device__ __forceinline__ float horizontal2(const SdfParams &p, int a, int b)
{
    const float rx = a > 0 ? a * p.dxf : (a < -1 ? -(a + 1) * p.dxf : 0.0f);
    const float ry = b > 0 ? b * p.dyf : (b < -1 ? -(b + 1) * p.dyf : 0.0f);
    return rx * rx + ry * ry;
}

// The FP32 distance of cell e of the window, or +inf when its lower bound (the
// horizontal gap and the vertical gap to its height range) exceeds lim.
template <bool TILE>
__device__ __forceinline__ float cell_f(const SdfParams &p, const Heights<TILE> &H, int a, int b, float rh2, float zf,
                                        float lim)
{
    const float e00 = H.f(a, b) - zf, e10 = H.f(a + 1, b) - zf;
    const float e01 = H.f(a, b + 1) - zf, e11 = H.f(a + 1, b + 1) - zf;
    const float gap = fmaxf(fmaxf(-fmaxf(fmaxf(e00, e10), fmaxf(e01, e11)), fminf(fminf(e00, e10), fminf(e01, e11))),
                            0.0f);
    if (rh2 + gap * gap > lim * lim) return INFINITY;
    return sqrtf(cell2<float>(a * p.dxf, b * p.dyf, p.dxf, p.dyf, p.rdxf, p.rdyf, e00, e10, e01, e11));
}

// Squared distance from node (i, j, z) to the surface, exact in FP64 for the
// nearest point within the window (else vert^2 or more).  On this part FP64 runs
// at a small fraction of the FP32 rate, so a first pass finds, in FP32, the
// smallest distance m over the window's cells (and the vertex straight below or
// above, |vert|); a second pass repeats the FP32 distances and evaluates in FP64
// only the cells within m + tol, tol a bound on twice the FP32 error (rounding of
// the heights, of z, of the coordinates, and of the arithmetic, each some ulps of
// the largest magnitude in play).  The cell holding the nearest point is always
// among them, so the result is the FP64 distance.
template <bool TILE>
__device__ double distance2(const SdfParams &p, const Heights<TILE> &H, double z, double vert, float tol)
{
    const float zf = (float)z;
    float m = fabsf((float)vert);
    for (int e = 0; e < p.ncells; ++e) {
        const int a = p.ca[e], b = p.cb[e];
        const float rh2 = horizontal2(p, a, b);
        const float lim = m + tol;
        if (rh2 > lim * lim) break;
        m = fminf(m, cell_f(p, H, a, b, rh2, zf, lim));
    }
    const float lim = m + tol;
    double best2 = vert * vert;
    for (int e = 0; e < p.ncells; ++e) {
        const int a = p.ca[e], b = p.cb[e];
        const float rh2 = horizontal2(p, a, b);
        if (rh2 > lim * lim) break;
        if (!(cell_f(p, H, a, b, rh2, zf, lim) <= lim)) continue;
        const double e00 = __dsub_rn(H.d(a, b), z), e10 = __dsub_rn(H.d(a + 1, b), z);
        const double e01 = __dsub_rn(H.d(a, b + 1), z), e11 = __dsub_rn(H.d(a + 1, b + 1), z);
        best2 = fmin(best2, cell2<double>(a * p.dx, b * p.dy, p.dx, p.dy, p.rdx, p.rdy, e00, e10, e01, e11));
    }
    return best2;
}

// z of level k on the uv-grid (g = 0) or the w-grid (g = 1), rounded once, as written
__device__ __forceinline__ double level_z(const SdfParams &p, int g, int k)
{
    return __dmul_rn(k + (g ? 0.0 : 0.5), p.dz);
}

// A block owns one row segment of 32 columns; its 8 warps share them, warp q
// taking levels q, q + 8, ... of each, so that the costly levels of a steep
// column spread over eight warps and every warp's store covers 32 consecutive
// nodes.  ZTAB: the levels' z sit in a shared table (2 nz doubles), so that a
// level outside the reach costs one subtraction and a store.  TILE: the heights
// the segment's windows touch sit in shared tiles, in FP64 and in FP32.
template <bool ZTAB, bool TILE>
__global__ void __launch_bounds__(kSdfCols * kSdfLanes) k_heightfield_sdf(const __grid_constant__ SdfParams p)
{
    extern __shared__ double smem[];
    __shared__ double part_min[kSdfLanes][kSdfCols], part_max[kSdfLanes][kSdfCols];
    double *const ztab = smem;
    double *const dtile = smem + (ZTAB ? 2 * p.nz : 0);
    const int th = 2 * p.wy + 1;
    float *const ftile = reinterpret_cast<float *>(dtile + (TILE ? th * p.tw : 0));
    const int seg = blockIdx.x % p.segs, j = blockIdx.x / p.segs;
    const int i_first = seg * kSdfCols;
    if (ZTAB) {
        for (int q = threadIdx.x; q < 2 * p.nz; q += kSdfCols * kSdfLanes) ztab[q] = level_z(p, q >= p.nz, q % p.nz);
    }
    if (TILE) {
        for (int q = threadIdx.x; q < th * p.tw; q += kSdfCols * kSdfLanes) {
            const int r = q / p.tw, cc = q % p.tw;
            const double v = __ldg(p.h + (int64_t)wrap_index(j - p.wy + r, p.ny) * p.nx +
                                   wrap_index(i_first - p.wx + cc, p.nx));
            dtile[q] = v;
            ftile[q] = (float)v;
        }
        __syncthreads();
    }
    const int c = threadIdx.x % kSdfCols, lane = threadIdx.x / kSdfCols;
    const int i = i_first + c;
    const bool live = i < p.nx;
    const Heights<TILE> H{p, dtile, ftile, c, live ? i : 0, j};
    // height range of every vertex a window cell touches, the window's rows
    // shared out over the lanes
    double lo = INFINITY, hi = -INFINITY;
    if (live) {
        for (int b = -p.wy + lane; b <= p.wy; b += kSdfLanes)
            for (int a = -p.wx; a <= p.wx; ++a) {
                const double q = H.d(a, b);
                lo = fmin(lo, q);
                hi = fmax(hi, q);
            }
    }
    part_min[lane][c] = lo;
    part_max[lane][c] = hi;
    __syncthreads();
    if (!live) return;
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int64_t col = (int64_t)j * p.nx + i;
    const double hv = H.d(0, 0);
    double hmin = hv, hmax = hv;
    for (int q = 0; q < kSdfLanes; ++q) {
        hmin = fmin(hmin, part_min[q][c]);
        hmax = fmax(hmax, part_max[q][c]);
    }
    const bool top = hv >= hmax, bottom = hv <= hmin;
    const double rdz = 1.0 / p.dz;
    // FP32 error allowance of the first pass (see distance2): 1e-5 of the largest
    // magnitudes involved, about 170 ulps
    const float scale = 2.0f * fmaxf(fabsf((float)hmin), fabsf((float)hmax)) + p.spanf;
    for (int g = 0; g < 2; ++g) {
        double *const out = g ? p.phi_w : p.phi_uv;
        const double off = g ? 0.0 : 0.5;
        // levels with hmin - reach <= z <= hmax + reach, widened by one level on
        // each side against rounding: only these can lie within the reach (a level
        // taken in needlessly still gets z - h, as its distance exceeds the reach)
        const double flo = fmin(fmax(floor((hmin - p.reach) * rdz - off) - 1.0, 0.0), (double)p.nz);
        const double fhi = fmin(fmax(ceil((hmax + p.reach) * rdz - off) + 1.0, -1.0), (double)(p.nz - 1));
        const int klo = (int)flo, khi = (int)fhi;
        for (int k = lane; k < p.nz; k += kSdfLanes) {
            // a level outside [klo, khi] costs one FP64 subtraction (FP64 is the
            // scarce unit here): the tests below are integer ones
            const double z = ZTAB ? ztab[g * p.nz + k] : level_z(p, g, k);
            const double vert = __dsub_rn(z, hv);
            double phi = vert;
            if (k >= klo && k <= khi) {
                // the column's own vertex is the nearest surface point when it is the
                // highest of the window and the node lies above it (every other surface
                // point is lower, so farther), or the lowest with the node below it
                const bool above = __double_as_longlong(vert) >= 0;
                if (!(above ? top : bottom)) {
                    const float tol = 1e-5f * (scale + 2.0f * fabsf((float)z));
                    const double d = sqrt(distance2(p, H, z, vert, tol));
                    if (d <= p.reach) phi = copysign(d, vert);
                }
            }
            out[k * plane + col] = phi;
        }
    }
}

}  // namespace

extern "C" int wmibm_heightfield_sdf(const wmibm_grid *g, const double *height, double reach, double *phi_uv,
                                     double *phi_w, void *stream)
{
    ApiRange nvtx_range("wmibm_heightfield_sdf");
    if (!g || !height || !phi_uv || !phi_w) return set_error(nullptr, WMIBM_EINVAL, "NULL grid or field pointer");
    if (g->nx < 1 || g->ny < 1 || g->nz < 3) return set_error(nullptr, WMIBM_EINVAL, "bad grid sizes");
    const int64_t n = (int64_t)g->nx * g->ny * g->nz;
    if (n >= ((int64_t)1 << 31)) return set_error(nullptr, WMIBM_EINVAL, "nx*ny*nz must be < 2^31");
    if (!(g->lx > 0.0) || !(g->ly > 0.0) || !(g->lz > 0.0) || !std::isfinite(g->lx) || !std::isfinite(g->ly) ||
        !std::isfinite(g->lz))
        return set_error(nullptr, WMIBM_EINVAL, "domain lengths must be finite and > 0");
    if (!(reach > 0.0) || !std::isfinite(reach)) return set_error(nullptr, WMIBM_EINVAL, "reach must be finite and > 0");
    if (phi_uv == phi_w) return set_error(nullptr, WMIBM_EINVAL, "phi_uv and phi_w must be distinct");
    SdfParams p = {};
    p.h = height;
    p.phi_uv = phi_uv;
    p.phi_w = phi_w;
    p.nx = g->nx;
    p.ny = g->ny;
    p.nz = g->nz;
    p.dx = g->lx / g->nx;
    p.dy = g->ly / g->ny;
    p.dz = g->lz / (g->nz - 1);
    p.rdx = 1.0 / p.dx;
    p.rdy = 1.0 / p.dy;
    p.reach = reach;
    const double wxd = std::ceil(reach / p.dx), wyd = std::ceil(reach / p.dy);
    if (wxd * wyd * 4.0 > kSdfMaxCells || wxd > 64 || wyd > 64)
        return set_error(nullptr, WMIBM_EINVAL,
                         "reach spans %.0f x %.0f cells; at most %d window cells and 128 in each direction", 2 * wxd,
                         2 * wyd, kSdfMaxCells);
    p.wx = (int32_t)wxd;
    p.wy = (int32_t)wyd;
    // window cells a in [-wx, wx - 1], b in [-wy, wy - 1]: every cell that meets
    // the disc of radius reach around the column; nearest (horizontally) first
    struct Cell {
        double r2;
        int a, b;
    };
    std::vector<Cell> cells;
    for (int b = -p.wy; b < p.wy; ++b)
        for (int a = -p.wx; a < p.wx; ++a) {
            const double rx = a > 0 ? a * p.dx : (a < -1 ? -(a + 1) * p.dx : 0.0);
            const double ry = b > 0 ? b * p.dy : (b < -1 ? -(b + 1) * p.dy : 0.0);
            const double r2 = rx * rx + ry * ry;
            if (r2 <= reach * reach * (1.0 + 1e-12)) cells.push_back({r2, a, b});
        }
    std::stable_sort(cells.begin(), cells.end(), [](const Cell &l, const Cell &r) { return l.r2 < r.r2; });
    p.ncells = (int32_t)cells.size();
    for (size_t e = 0; e < cells.size(); ++e) {
        p.ca[e] = (int8_t)cells[e].a;
        p.cb[e] = (int8_t)cells[e].b;
    }
    p.segs = (g->nx + kSdfCols - 1) / kSdfCols;
    p.tw = kSdfCols + 2 * p.wx;
    p.dxf = (float)p.dx;
    p.dyf = (float)p.dy;
    p.rdxf = (float)(1.0 / p.dx);
    p.rdyf = (float)(1.0 / p.dy);
    p.spanf = (float)((p.wx + 1) * p.dx + (p.wy + 1) * p.dy);
    const int64_t blocks = (int64_t)p.segs * g->ny;
    if (blocks >= ((int64_t)1 << 31)) return set_error(nullptr, WMIBM_EINVAL, "too many row segments");
    const size_t zbytes = (size_t)2 * g->nz * sizeof(double);
    const size_t tbytes = (size_t)(2 * p.wy + 1) * p.tw * (sizeof(double) + sizeof(float));
    const bool ztab = zbytes <= (size_t)kSdfSmemCap, tile = tbytes <= (size_t)kSdfSmemCap;
    const size_t smem = (ztab ? zbytes : 0) + (tile ? tbytes : 0);
    const dim3 grid((unsigned)blocks), block(kSdfCols * kSdfLanes);
    cudaStream_t st = (cudaStream_t)stream;
    if (ztab && tile)
        k_heightfield_sdf<true, true><<<grid, block, smem, st>>>(p);
    else if (ztab)
        k_heightfield_sdf<true, false><<<grid, block, smem, st>>>(p);
    else if (tile)
        k_heightfield_sdf<false, true><<<grid, block, smem, st>>>(p);
    else
        k_heightfield_sdf<false, false><<<grid, block, smem, st>>>(p);
    return cuda_status(nullptr, cudaGetLastError(), "k_heightfield_sdf launch");
}
