// Bulk-copy (TMA) pipelined stencil for f = -div(tau) (Eq. 2, Eq. 18, Eqs. 15-16
// of Liu & Stevens, arXiv:2006.03343), and the fused per-step kernel built on it.
//
// Stencil: the grid is cut into strips of TY full x-rows (j0 .. j0+TY-1) and the
// (strip, level) units are split evenly over a persistent grid (one contiguous
// range of units per block; a range spans at most a few strip segments).  Per
// block, lane 0 of warp 0 is the producer: it issues 1D bulk copies of the rows
// a stage needs into a ring of S shared-memory stages and arms the stage's
// "full" mbarrier with the byte count.  A stage at level k holds
//   txx, tzz at k (TY rows), txy, tyy at k (TY + 2 rows: y-halo),
//   txz at k+1 (TY rows), tyz at k+1 (TY + 2 rows)
// and the stage before it supplies txz, tyz at k and tzz at k-1, so every
// stress row is fetched from HBM once per strip.  A segment starts with a
// prologue stage that holds only tzz at k-1 and txz, tyz at k.  Consumer warps
// form f for the TY rows, with x-neighbours from warp shuffles and periodic
// wrap inside the staged full rows, and release the stage through the "empty"
// mbarrier.
//
// Fused step (two kernels chained by programmatic dependent launch): the wall
// kernel evaluates the wall model of Sec. 3.3 at every band node and zeroes the
// solid runs (stresses written to the caller's arrays, band statistics reduced
// on the way) and lets the stencil kernel launch at once.  The stencil kernel
// first streams its "clean" stages, whose rows hold no band or solid node;
// before its first "dirty" stage, and before the body mask of Eq. 27 (which may
// change the velocity only after every band stencil has read it), it waits on
// the grid dependency, i.e. for the wall kernel to have completed.
//
// Every mbarrier wait is bounded: on time-out the kernel records a status code
// in device memory and leaves its loops.
#include <algorithm>

#include "band.cuh"
#include "tma.cuh"

using namespace wmibm;

namespace {


template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    static constexpr int V = 4;
    using vec = float4;
};
template <>
struct VecOf<double> {
    static constexpr int V = 2;
    using vec = double2;
};

template <typename T>
struct Pack {
    T v[VecOf<T>::V];
};

__device__ __forceinline__ Pack<float> lds(const float *p)
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    return Pack<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Pack<double> lds(const double *p)
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    return Pack<double>{{a.x, a.y}};
}
__device__ __forceinline__ void stg(float *p, const Pack<float> &x)
{
    *reinterpret_cast<float4 *>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
__device__ __forceinline__ void stg(double *p, const Pack<double> &x)
{
    *reinterpret_cast<double2 *>(p) = make_double2(x.v[0], x.v[1]);
}

template <typename T>
struct StencilParams {
    const T *tau[6];          // txx txy tyy tzz txz tyz
    T *f[3];
    int32_t nx, ny, nz, nstrips;
    int64_t units;            // nstrips * nz
    T cx, cy, cz;
    int stages, ncons, nwall;
    int32_t da, db;           // dirty levels (units whose stages depend on the wall phase)
    uint32_t stage_elems;
    int *status;
    // fused step: phase 1 (wall model, solid zeros) and the body mask
    void *u, *v, *w;
    const void *rec;
    int64_t nb_w, nb_uv;
    const int2 *runs_w, *runs_uv;   // solid runs along x (first node, length)
    int64_t nr_w, nr_uv;
    int do_mask;
    const int32_t *body_w, *body_uv;
    int64_t nbody_w, nbody_uv;
    const T *gpx, *gpy, *gpz;
    T mask_c;                 // 3 dt / 2
    T *partials;
    unsigned *ticket;
    wmibm_band_stats *stats;
    const T *logz0;
    T log_phi_c, kappa2;
};

// The units (strip s, level k) are split into "clean" units, whose stage rows
// (levels k-1 .. k+1) hold no band or solid node, and "dirty" units (levels
// [da, db)).  Clean units do not depend on the wall-model phase of the fused
// kernel, so every block streams its share of clean units first and only then
// its share of dirty units.
struct Schedule {
    int64_t c0, c1, d0, d1;   // this block's ranges in the clean and dirty unit spaces
    int32_t nz, da, db;       // dirty levels [da, db)
};

__device__ __forceinline__ Schedule block_schedule(int32_t nstrips, int32_t nz, int32_t da, int32_t db)
{
    Schedule sc;
    const int64_t C = (int64_t)nstrips * (da + (nz - db));
    const int64_t D = (int64_t)nstrips * (db - da);
    sc.c0 = C * blockIdx.x / gridDim.x;
    sc.c1 = C * (blockIdx.x + 1) / gridDim.x;
    sc.d0 = D * blockIdx.x / gridDim.x;
    sc.d1 = D * (blockIdx.x + 1) / gridDim.x;
    sc.nz = nz;
    sc.da = da;
    sc.db = db;
    return sc;
}

// Sequence of stages a block processes: its clean units then its dirty units,
// cut into segments of consecutive levels of one strip; each segment starts
// with a prologue stage followed by one main stage per level.
struct StageIter {
    Schedule sc;
    int64_t idx;
    int phase;                // 0 clean, 1 dirty, 2 done
    int32_t s, k;
    bool prologue, done, dirty;
    __device__ void unit(int ph, int64_t i, int32_t &s_, int32_t &k_) const
    {
        if (ph == 0) {
            const int32_t lc = sc.da + (sc.nz - sc.db);
            s_ = (int32_t)(i / lc);
            const int32_t r = (int32_t)(i - (int64_t)s_ * lc);
            k_ = r < sc.da ? r : sc.db + (r - sc.da);
        } else {
            const int32_t ld = sc.db - sc.da;
            s_ = (int32_t)(i / ld);
            k_ = sc.da + (int32_t)(i - (int64_t)s_ * ld);
        }
    }
    __device__ void settle()
    {
        while (phase < 2 && idx >= (phase == 0 ? sc.c1 : sc.d1)) {
            ++phase;
            idx = sc.d0;
        }
        done = phase >= 2;
        if (!done) {
            unit(phase, idx, s, k);
            prologue = true;
            dirty = phase == 1;
        }
    }
    __device__ void init(const Schedule &s_)
    {
        sc = s_;
        phase = 0;
        idx = sc.c0;
        settle();
    }
    __device__ void next()
    {
        if (prologue) {
            prologue = false;
            return;
        }
        ++idx;
        if (idx < (phase == 0 ? sc.c1 : sc.d1)) {
            int32_t s2, k2;
            unit(phase, idx, s2, k2);
            prologue = !(s2 == s && k2 == k + 1);
            s = s2;
            k = k2;
            return;
        }
        settle();
    }
};

template <int TY>
struct Slots {
    static constexpr int XX = 0;
    static constexpr int XY = TY;
    static constexpr int YY = 2 * TY + 2;
    static constexpr int ZZ = 3 * TY + 4;
    static constexpr int XZ = 4 * TY + 4;
    static constexpr int YZ = 5 * TY + 4;
    static constexpr int ROWS = 6 * TY + 6;
};

__device__ __forceinline__ int32_t wrapj(int32_t j, int32_t ny) { return j < 0 ? j + ny : (j >= ny ? j - ny : j); }

// ------------------------------------------------------------------------- //
// producer: lane 0 of warp 0
// ------------------------------------------------------------------------- //
// Waits until the preceding kernel of the stream (the wall kernel) has
// completed and its writes are visible (programmatic dependent launch; without
// a programmatic dependency the stream order already guarantees it).
__device__ __forceinline__ void wait_wall_kernel()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename T, int TY, bool FUSED>
__device__ void produce(const StencilParams<T> &p, T *data, uint64_t *full, uint64_t *empty, const Schedule &sc)
{
    using S_ = Slots<TY>;
    const int32_t nx = p.nx, ny = p.ny;
    const uint32_t row_bytes = (uint32_t)nx * sizeof(T);
    const int64_t plane = (int64_t)nx * ny;
    const T *const txx = p.tau[0], *const txy = p.tau[1], *const tyy = p.tau[2];
    const T *const tzz = p.tau[3], *const txz = p.tau[4], *const tyz = p.tau[5];
    uint32_t g = 0;
    bool released = !FUSED;
    StageIter it;
    for (it.init(sc); !it.done; it.next(), ++g) {
        const int b = (int)(g % (uint32_t)p.stages);
        if (g >= (uint32_t)p.stages) {
            if (!mbar_wait(&empty[b], ((g / p.stages) & 1u) ^ 1u, p.status, kDevStatusEmptyTimeout)) break;
        }
        if (it.dirty && !released) {
            // the stresses written by the wall kernel must be complete and visible
            // to the bulk copies (async proxy) before a dirty stage
            wait_wall_kernel();
            asm volatile("fence.proxy.async.global;" ::: "memory");
            released = true;
        }
        T *st = data + (size_t)b * p.stage_elems;
        const int32_t j0 = it.s * TY;
        const int32_t k = it.k;
        // rows [jstart, jstart + cnt) of one level (periodic in j) into consecutive
        // slot rows: one bulk copy per contiguous piece (two where the interval wraps)
        auto issue = [&](const T *arr, int32_t lev, int32_t jstart, int32_t cnt, int32_t slot) {
            const T *base = arr + (int64_t)lev * plane;
            T *dst = st + (size_t)slot * nx;
            if (jstart < 0) {
                bulk_g2s(dst, base + (int64_t)(ny - 1) * nx, row_bytes, &full[b]);
                bulk_g2s(dst + nx, base, (uint32_t)(cnt - 1) * row_bytes, &full[b]);
            } else if (jstart + cnt > ny) {
                const int32_t first = ny - jstart;
                bulk_g2s(dst, base + (int64_t)jstart * nx, (uint32_t)first * row_bytes, &full[b]);
                bulk_g2s(dst + (size_t)first * nx, base, (uint32_t)(cnt - first) * row_bytes, &full[b]);
            } else {
                bulk_g2s(dst, base + (int64_t)jstart * nx, (uint32_t)cnt * row_bytes, &full[b]);
            }
        };
        if (it.prologue) {
            const uint32_t rows = (k > 0 ? TY : 0) + TY + (TY + 2);
            mbar_arrive_expect_tx(&full[b], rows * row_bytes);
            if (k > 0) issue(tzz, k - 1, j0, TY, S_::ZZ);
            issue(txz, k, j0, TY, S_::XZ);
            issue(tyz, k, j0 - 1, TY + 2, S_::YZ);
        } else {
            const bool up = k + 1 < p.nz;
            const uint32_t rows = TY + 2 * (TY + 2) + TY + (up ? TY + (TY + 2) : 0);
            mbar_arrive_expect_tx(&full[b], rows * row_bytes);
            issue(txx, k, j0, TY, S_::XX);
            issue(txy, k, j0 - 1, TY + 2, S_::XY);
            issue(tyy, k, j0 - 1, TY + 2, S_::YY);
            issue(tzz, k, j0, TY, S_::ZZ);
            if (up) {
                issue(txz, k + 1, j0, TY, S_::XZ);
                issue(tyz, k + 1, j0 - 1, TY + 2, S_::YZ);
            }
        }
    }
    if (!it.done) {
        // gave up: let the copies already issued land before the block exits
        const uint32_t first = g > (uint32_t)p.stages ? g - p.stages : 0;
        for (uint32_t q = first; q < g; ++q)
            mbar_wait(&full[q % p.stages], (q / p.stages) & 1u, p.status, kDevStatusFullTimeout);
    }
}

// ------------------------------------------------------------------------- //
// consumers: f for the TY rows of a main stage
// ------------------------------------------------------------------------- //
template <typename T, int TY>
__device__ void consume_level(const StencilParams<T> &p, const T *cur, const T *prv, int32_t k, int32_t j0, int cw,
                              int lane)
{
    using S_ = Slots<TY>;
    constexpr int V = VecOf<T>::V;
    const int32_t nx = p.nx;
    const int nq = nx / V;
    const int groups = TY * nq;
    const int64_t plane = (int64_t)nx * p.ny;
    const bool top = (k == p.nz - 1);
    const bool bottom = (k == 0);
    for (int base = cw * 32; base < groups; base += p.ncons * 32) {
        const int gi = base + lane;
        const bool valid = gi < groups;
        const int gc = valid ? gi : groups - 1;
        const int r = gc / nq, q = gc - r * nq;
        const int i = q * V;
        const int64_t o = (int64_t)k * plane + (int64_t)(j0 + r) * nx + i;
        Pack<T> Fx, Fy, Fz;
        if (top) {
            for (int e = 0; e < V; ++e) {
                Fx.v[e] = T(0);
                Fy.v[e] = T(0);
                Fz.v[e] = T(0);
            }
        } else {
            const int im = (i == 0) ? nx - 1 : i - 1;
            const int ip = (i + V == nx) ? 0 : i + V;
            const T *XXr = cur + (S_::XX + r) * nx;
            const T *XYc = cur + (S_::XY + r + 1) * nx;
            const T *XZ0 = prv + (S_::XZ + r) * nx;
            const Pack<T> xx = lds(XXr + i);
            const Pack<T> xy = lds(XYc + i);
            const Pack<T> xym = lds(cur + (S_::XY + r) * nx + i), xyp = lds(cur + (S_::XY + r + 2) * nx + i);
            const Pack<T> yym = lds(cur + (S_::YY + r) * nx + i), yyp = lds(cur + (S_::YY + r + 2) * nx + i);
            const Pack<T> zz = lds(cur + (S_::ZZ + r) * nx + i);
            const Pack<T> xz1 = lds(cur + (S_::XZ + r) * nx + i);
            const Pack<T> yz1 = lds(cur + (S_::YZ + r + 1) * nx + i);
            const Pack<T> xz0 = lds(XZ0 + i);
            const Pack<T> yz0 = lds(prv + (S_::YZ + r + 1) * nx + i);
            const Pack<T> yz0m = lds(prv + (S_::YZ + r) * nx + i), yz0p = lds(prv + (S_::YZ + r + 2) * nx + i);
            Pack<T> zzm;
            if (!bottom)
                zzm = lds(prv + (S_::ZZ + r) * nx + i);
            else
                for (int e = 0; e < V; ++e) zzm.v[e] = T(0);
            // x-neighbours at the vector edges: from the adjacent lane when it holds
            // the adjacent vector of the same row, else from shared memory
            const unsigned full_mask = 0xffffffffu;
            T xxl = __shfl_up_sync(full_mask, xx.v[V - 1], 1), xxr = __shfl_down_sync(full_mask, xx.v[0], 1);
            T xyl = __shfl_up_sync(full_mask, xy.v[V - 1], 1), xyr = __shfl_down_sync(full_mask, xy.v[0], 1);
            T xzl = __shfl_up_sync(full_mask, xz0.v[V - 1], 1), xzr = __shfl_down_sync(full_mask, xz0.v[0], 1);
            const bool left_ok = lane > 0 && q > 0;
            const bool right_ok = lane < 31 && q < nq - 1 && gi + 1 < groups;
            if (!left_ok) {
                xxl = XXr[im];
                xyl = XYc[im];
                xzl = XZ0[im];
            }
            if (!right_ok) {
                xxr = XXr[ip];
                xyr = XYc[ip];
                xzr = XZ0[ip];
            }
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const T xxm_ = e == 0 ? xxl : xx.v[e - 1], xxp_ = e == V - 1 ? xxr : xx.v[e + 1];
                const T xym_ = e == 0 ? xyl : xy.v[e - 1], xyp_ = e == V - 1 ? xyr : xy.v[e + 1];
                const T xzm_ = e == 0 ? xzl : xz0.v[e - 1], xzp_ = e == V - 1 ? xzr : xz0.v[e + 1];
                Fx.v[e] = -((xxp_ - xxm_) * p.cx + (xyp.v[e] - xym.v[e]) * p.cy + (xz1.v[e] - xz0.v[e]) * p.cz);
                Fy.v[e] = -((xyp_ - xym_) * p.cx + (yyp.v[e] - yym.v[e]) * p.cy + (yz1.v[e] - yz0.v[e]) * p.cz);
                const T fz = -((xzp_ - xzm_) * p.cx + (yz0p.v[e] - yz0m.v[e]) * p.cy + (zz.v[e] - zzm.v[e]) * p.cz);
                Fz.v[e] = bottom ? T(0) : fz;
            }
        }
        if (valid) {
            stg(p.f[0] + o, Fx);
            stg(p.f[1] + o, Fy);
            stg(p.f[2] + o, Fz);
        }
    }
}

template <typename T, int TY>
__device__ void consume(const StencilParams<T> &p, const T *data, uint64_t *ready, uint64_t *empty,
                        const Schedule &sc, int cw, int lane)
{
    uint32_t g = 0;
    int prevb = -1;
    StageIter it;
    for (it.init(sc); !it.done; it.next(), ++g) {
        const int b = (int)(g % (uint32_t)p.stages);
        if (!mbar_wait(&ready[b], (g / p.stages) & 1u, p.status, kDevStatusFullTimeout)) break;
        if (!it.prologue)
            consume_level<T, TY>(p, data + (size_t)b * p.stage_elems, data + (size_t)prevb * p.stage_elems, it.k,
                                 it.s * TY, cw, lane);
        if (prevb >= 0) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[prevb]);
        }
        prevb = b;
    }
}

// ------------------------------------------------------------------------- //
// fused step: phase 1, grid barrier, mask
// ------------------------------------------------------------------------- //

// Wall phase: the participating threads of the whole grid share the band
// records (two per thread and round, all loads issued before the stores) and
// then the solid runs (a warp zeroes one run at a time with coalesced stores,
// run descriptors fetched 32 at a time).
template <typename T, typename VEL>
__device__ void wall_phase(const StencilParams<T> &p, T *acc, int wt, int nthreads)
{
    // let the stencil kernel (next in the stream) launch right away
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    T *const oxx = const_cast<T *>(p.tau[0]), *const oxy = const_cast<T *>(p.tau[1]);
    T *const oyy = const_cast<T *>(p.tau[2]), *const ozz = const_cast<T *>(p.tau[3]);
    T *const oxz = const_cast<T *>(p.tau[4]), *const oyz = const_cast<T *>(p.tau[5]);
    const VEL *const vu = reinterpret_cast<const VEL *>(p.u);
    const VEL *const vv = reinterpret_cast<const VEL *>(p.v);
    const VEL *const vw = reinterpret_cast<const VEL *>(p.w);
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int64_t nrec = p.nb_w + p.nb_uv;
    const int64_t stride = (int64_t)gridDim.x * nthreads;
    const int64_t tid = (int64_t)blockIdx.x * nthreads + wt;

    auto store = [&](const BandOut<T> &o, bool is_w) {
        if (is_w) {
            oxz[o.idx] = o.t0;
            oyz[o.idx] = o.t1;
        } else {
            oxx[o.idx] = o.t0;
            oxy[o.idx] = o.t1;
            oyy[o.idx] = o.t2;
            ozz[o.idx] = o.t3;
        }
        stats_add(acc, is_w ? 0 : 1, o.tw, o.ur);
    };
    for (int64_t t0 = tid; t0 < nrec; t0 += 2 * stride) {
        const int64_t t1 = t0 + stride;
        BandOut<T> a, b;
        a = band_model<T, VEL>(p.rec, t0, t0 < p.nb_w, vu, vv, vw, p.nx, p.ny, plane, p.logz0, p.log_phi_c,
                               p.kappa2);
        if (t1 < nrec)
            b = band_model<T, VEL>(p.rec, t1, t1 < p.nb_w, vu, vv, vw, p.nx, p.ny, plane, p.logz0, p.log_phi_c,
                                   p.kappa2);
        store(a, t0 < p.nb_w);
        if (t1 < nrec) store(b, t1 < p.nb_w);
    }

    // solid nodes: the stress is set to zero (Sec. 3.3)
    const int lane = wt & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (nthreads / 32);
    const int64_t gw = (int64_t)blockIdx.x * (nthreads / 32) + (wt >> 5);
    const int64_t nruns = p.nr_w + p.nr_uv;
    // warp gw takes runs gw, gw + nwarps, ...: lane q fetches the descriptor of
    // the q-th of them, then the warp zeroes them one after the other
    for (int64_t base = gw; base < nruns; base += nwarps * 32) {
        const int64_t t = base + (int64_t)lane * nwarps;
        int2 run = make_int2(0, 0);
        if (t < nruns) run = __ldg(t < p.nr_w ? p.runs_w + t : p.runs_uv + (t - p.nr_w));
        const int nq = (int)min((int64_t)32, (nruns - base + nwarps - 1) / nwarps);
        for (int q = 0; q < nq; ++q) {
            const int32_t start = __shfl_sync(0xffffffffu, run.x, q);
            const int32_t len = __shfl_sync(0xffffffffu, run.y, q);
            const bool is_w = base + (int64_t)q * nwarps < p.nr_w;
            for (int32_t x = lane; x < len; x += 32) {
                const int64_t idx = (int64_t)start + x;
                if (is_w) {
                    oxz[idx] = T(0);
                    oyz[idx] = T(0);
                } else {
                    oxx[idx] = T(0);
                    oxy[idx] = T(0);
                    oyy[idx] = T(0);
                    ozz[idx] = T(0);
                }
            }
        }
    }
}

// Eq. 27: body velocity = 3 dt/2 grad p, or 0 (grid-stride over the body lists).
template <typename T, typename VEL>
__device__ void mask_phase(const StencilParams<T> &p, int64_t tid, int64_t stride)
{
    VEL *const vu = reinterpret_cast<VEL *>(p.u);
    VEL *const vv = reinterpret_cast<VEL *>(p.v);
    VEL *const vw = reinterpret_cast<VEL *>(p.w);
    for (int64_t t = tid; t < p.nbody_uv; t += stride) {
        const int32_t idx = __ldg(p.body_uv + t);
        vu[idx] = to_vel<VEL, T>(p.gpx ? p.mask_c * __ldg(p.gpx + idx) : T(0));
        vv[idx] = to_vel<VEL, T>(p.gpy ? p.mask_c * __ldg(p.gpy + idx) : T(0));
    }
    for (int64_t t = tid; t < p.nbody_w; t += stride) {
        const int32_t idx = __ldg(p.body_w + t);
        vw[idx] = to_vel<VEL, T>(p.gpz ? p.mask_c * __ldg(p.gpz + idx) : T(0));
    }
}

template <typename T, typename VEL>
__global__ void __launch_bounds__(256) k_wall(StencilParams<T> p)
{
    __shared__ T red[32][kStatVals];
    T acc[kStatVals];
    stats_identity(acc);
    wall_phase<T, VEL>(p, acc, threadIdx.x, blockDim.x);
    if (p.stats) {
        stats_block_reduce(acc, red);
        stats_finish(acc, red, p.partials, p.ticket, gridDim.x, p.stats, p.nb_w, p.nb_uv);
    }
}

template <typename T, typename VEL, int TY, bool FUSED>
__global__ void __launch_bounds__(512) k_stencil(StencilParams<T> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + 8;
    T *data = reinterpret_cast<T *>(smem_raw + 256);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < p.stages; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], p.ncons);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const Schedule sc = block_schedule(p.nstrips, p.nz, FUSED ? p.da : 0, FUSED ? p.db : 0);

    if (warp == 0) {
        // producer: clean stages right away (their rows are not written by the
        // wall kernel), dirty stages once the wall kernel has completed
        if (lane == 0) produce<T, TY, FUSED>(p, data, full, empty, sc);
        __syncwarp();
    } else {
        consume<T, TY>(p, data, full, empty, sc, warp - 1, lane);
        if (FUSED && p.do_mask) {
            wait_wall_kernel();
            const int nct = p.ncons * 32;
            mask_phase<T, VEL>(p, (int64_t)blockIdx.x * nct + (threadIdx.x - 32), (int64_t)gridDim.x * nct);
        }
    }
}

template <typename T>
size_t stage_elems_for(int ty, int nx) { return (size_t)(6 * ty + 6) * nx; }

constexpr int kMaxDynSmem = 200 * 1024;

template <typename T, typename VEL, int TY, bool FUSED>
int launch_ty(wmibm_handle *h, StencilParams<T> &p, const StencilConfig &c, cudaStream_t stream, bool pdl)
{
    auto kern = k_stencil<T, VEL, TY, FUSED>;
    static bool attr_done = false;      // once per instantiation and process
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return cuda_status(h, e, "stencil smem attribute");
        attr_done = true;
    }
    const size_t smem = 256 + (size_t)c.stages * p.stage_elems * sizeof(T);
    const int threads = 32 * (1 + p.ncons);
    // occupancy of this shape, cached in the handle
    const int key = (FUSED ? 1 : 0) | (TY << 1) | (c.stages << 4) | (c.consumer_warps << 8) | (c.wall_warps << 12);
    int per_sm = 0;
    for (int q = 0; q < 8; ++q)
        if (h->occ_key[q] == key) per_sm = h->occ_val[q];
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return cuda_status(h, e, "stencil occupancy");
        if (per_sm < 1) return set_error(h, WMIBM_EINVAL, "stencil tile does not fit on an SM");
        const int slot = h->occ_next++ & 7;
        h->occ_key[slot] = key;
        h->occ_val[slot] = per_sm;
    }
    if (c.blocks_per_sm > 0 && c.blocks_per_sm < per_sm) per_sm = c.blocks_per_sm;
    int64_t grid = (int64_t)per_sm * h->sm_count;
    if (grid > p.units) grid = p.units;
    if (FUSED && pdl) {
        // programmatic dependent of the wall kernel launched just before
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cuda_status(h, cudaLaunchKernelEx(&cfg, kern, p), "k_stencil launch");
    }
    kern<<<(unsigned)grid, threads, smem, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_stencil launch");
}

bool aligned16(const void *q) { return ((uintptr_t)q & 15u) == 0; }

template <typename T>
void fill_params(wmibm_handle *h, StencilParams<T> &p, const void *const tau[6], void *const f[3], void *u, void *v,
                 void *w, wmibm_band_stats *stats, const void *logz0, const void *const gradp[3], int do_mask,
                 double dt, const StencilConfig &c);

template <typename T, typename VEL, bool FUSED>
int launch(wmibm_handle *h, const void *const tau[6], void *const f[3], void *u, void *v, void *w,
           wmibm_band_stats *stats, const void *logz0, const void *const gradp[3], int do_mask, double dt,
           const StencilConfig &c, cudaStream_t stream, bool pdl)
{
    StencilParams<T> p;
    fill_params<T>(h, p, tau, f, u, v, w, stats, logz0, gradp, do_mask, dt, c);
    switch (c.rows) {
    case 1: return launch_ty<T, VEL, 1, FUSED>(h, p, c, stream, pdl);
    case 2: return launch_ty<T, VEL, 2, FUSED>(h, p, c, stream, pdl);
    case 4: return launch_ty<T, VEL, 4, FUSED>(h, p, c, stream, pdl);
    default: return set_error(h, WMIBM_EINVAL, "stencil rows must be 1, 2 or 4");
    }
}

template <typename T>
void fill_params(wmibm_handle *h, StencilParams<T> &p, const void *const tau[6], void *const f[3], void *u, void *v,
                 void *w, wmibm_band_stats *stats, const void *logz0, const void *const gradp[3], int do_mask,
                 double dt, const StencilConfig &c)
{
    for (int a = 0; a < 6; ++a) p.tau[a] = (const T *)tau[a];
    for (int a = 0; a < 3; ++a) p.f[a] = (T *)f[a];
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz;
    p.nstrips = c.rows > 0 ? h->ny / c.rows : 0;
    p.units = (int64_t)p.nstrips * h->nz;
    p.cx = (T)(1.0 / (2.0 * h->dx));
    p.cy = (T)(1.0 / (2.0 * h->dy));
    p.cz = (T)(1.0 / h->dz);
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    p.nwall = c.wall_warps;
    p.da = h->dirty_lo;
    p.db = h->dirty_hi;
    p.stage_elems = (uint32_t)stage_elems_for<T>(c.rows > 0 ? c.rows : 1, h->nx);
    p.status = h->dev_status;
    p.u = u; p.v = v; p.w = w;
    p.rec = h->rec;
    p.nb_w = h->lists.n[WMIBM_LIST_BAND_W];
    p.nb_uv = h->lists.n[WMIBM_LIST_BAND_UV];
    p.runs_w = h->runs[0];
    p.runs_uv = h->runs[1];
    p.nr_w = h->nruns[0];
    p.nr_uv = h->nruns[1];
    p.do_mask = do_mask;
    p.body_w = h->lists.p[WMIBM_LIST_BODY_W];
    p.body_uv = h->lists.p[WMIBM_LIST_BODY_UV];
    p.nbody_w = h->lists.n[WMIBM_LIST_BODY_W];
    p.nbody_uv = h->lists.n[WMIBM_LIST_BODY_UV];
    p.gpx = gradp ? (const T *)gradp[0] : nullptr;
    p.gpy = gradp ? (const T *)gradp[1] : nullptr;
    p.gpz = gradp ? (const T *)gradp[2] : nullptr;
    p.mask_c = (T)(1.5 * dt);
    p.partials = (T *)h->partials;
    p.ticket = h->ticket;
    p.stats = stats;
    p.logz0 = (const T *)logz0;
    p.log_phi_c = (T)log(h->phi_c);
    p.kappa2 = (T)(h->kappa * h->kappa);
}

// The wall kernel: persistent grid sized by occupancy, wall_warps warps per block.
template <typename T, typename VEL>
int launch_wall(wmibm_handle *h, void *const tau[6], const void *u, const void *v, const void *w,
                wmibm_band_stats *stats, const void *logz0, cudaStream_t stream)
{
    StencilParams<T> p;
    StencilConfig c = {};
    void *const none[3] = {nullptr, nullptr, nullptr};
    fill_params<T>(h, p, (const void *const *)tau, none, const_cast<void *>(u), const_cast<void *>(v),
                   const_cast<void *>(w), stats, logz0, nullptr, 0, 0.0, c);
    const int wthreads = 32 * (h->tuning.wall_warps > 0 ? h->tuning.wall_warps : 8);
    int wper = 0;
    const int wkey = 0x100000 | wthreads | (sizeof(T) == 8 ? 0x200000 : 0);
    for (int q = 0; q < 8; ++q)
        if (h->occ_key[q] == wkey) wper = h->occ_val[q];
    if (wper == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, k_wall<T, VEL>, wthreads, 0);
        if (e != cudaSuccess) return cuda_status(h, e, "wall occupancy");
        if (wper < 1) wper = 1;
        const int slot = h->occ_next++ & 7;
        h->occ_key[slot] = wkey;
        h->occ_val[slot] = wper;
    }
    const int64_t wgrid = std::min<int64_t>((int64_t)wper * h->sm_count, h->partial_blocks);
    k_wall<T, VEL><<<(unsigned)wgrid, wthreads, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_wall launch");
}

}  // namespace

namespace wmibm {

// Chooses the stencil tile for this handle (or validates the one set by tuning).
// Returns false when the pipelined path cannot take this grid / these buffers.
bool stencil_config(const wmibm_handle *h, const void *const tau[6], void *const f[3], StencilConfig *out)
{
    const size_t es = elem_size(h->dtype);
    const int V = 16 / (int)es;
    if (h->tuning.force_path == 2) return false;
    if (h->nx % V != 0 || h->nz < 3) return false;
    for (int a = 0; a < 6; ++a)
        if (!aligned16(tau[a])) return false;
    for (int a = 0; a < 3; ++a)
        if (!aligned16(f[a])) return false;
    StencilConfig c;
    auto stage_bytes_of = [&](int rows) { return (size_t)(6 * rows + 6) * h->nx * es; };
    c.rows = h->tuning.rows;
    c.stages = h->tuning.stages;
    if (c.rows == 0) {
        // default: 2-row strips with at least 3 stages within ~110 KB of shared
        // memory (two or three blocks per SM); 1-row strips when rows are wide
        c.rows = (h->ny % 2 == 0 && h->ny >= 4) ? 2 : 1;
        if (c.rows == 2 && c.stages == 0 && 3 * stage_bytes_of(2) > 110 * 1024) c.rows = 1;
    }
    if (!(c.rows == 1 || c.rows == 2 || c.rows == 4)) return false;
    if (h->ny % c.rows != 0 || h->ny < c.rows + 2) return false;
    const size_t stage_bytes = stage_bytes_of(c.rows);
    if (c.stages == 0) {
        c.stages = 4;
        while (c.stages > 2 && (size_t)c.stages * stage_bytes > 110 * 1024) --c.stages;
    }
    if (c.stages < 2 || c.stages > 8) return false;
    if ((size_t)c.stages * stage_bytes + 256 > (size_t)kMaxDynSmem) return false;
    c.consumer_warps = h->tuning.consumer_warps > 0 ? h->tuning.consumer_warps : 4;
    c.wall_warps = h->tuning.wall_warps;
    if (1 + c.consumer_warps + c.wall_warps > 16) return false;
    c.blocks_per_sm = h->tuning.blocks_per_sm;
    *out = c;
    return true;
}

int stencil_force(wmibm_handle *h, const void *const tau[6], void *const f[3], const StencilConfig &c,
                  cudaStream_t stream)
{
    if (h->dtype == WMIBM_F64)
        return launch<double, double, false>(h, tau, f, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                                             0.0, c, stream, false);
    return launch<float, float, false>(h, tau, f, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0.0, c,
                                       stream, false);
}

// The pipelined stencil followed, in the same launch, by the body mask (Eq. 27).
// With pdl the launch is a programmatic dependent of the preceding kernel.
int stencil_force_mask(wmibm_handle *h, void *u, void *v, void *w, const void *const tau[6], void *const f[3],
                       const void *const gradp[3], double dt, const StencilConfig &c, bool pdl, cudaStream_t stream)
{
    if (h->dtype == WMIBM_F64)
        return launch<double, double, true>(h, tau, f, u, v, w, nullptr, nullptr, gradp, 1, dt, c, stream, pdl);
    if (h->vel_dtype == WMIBM_BF16)
        return launch<float, __nv_bfloat16, true>(h, tau, f, u, v, w, nullptr, nullptr, gradp, 1, dt, c, stream, pdl);
    return launch<float, float, true>(h, tau, f, u, v, w, nullptr, nullptr, gradp, 1, dt, c, stream, pdl);
}

// The wall kernel with caller-provided reduction scratch and grid size (used by
// the entry point whose scratch lives in a static device array).
int wall_model_with_scratch(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                            wmibm_band_stats *stats, void *partials, unsigned *ticket, unsigned blocks,
                            cudaStream_t stream)
{
    StencilConfig c = {};
    void *const none[3] = {nullptr, nullptr, nullptr};
    if (h->dtype == WMIBM_F64) {
        StencilParams<double> p;
        fill_params<double>(h, p, (const void *const *)tau, none, const_cast<void *>(u), const_cast<void *>(v),
                            const_cast<void *>(w), stats, nullptr, nullptr, 0, 0.0, c);
        p.partials = (double *)partials;
        p.ticket = ticket;
        k_wall<double, double><<<blocks, 256, 0, stream>>>(p);
    } else {
        StencilParams<float> p;
        fill_params<float>(h, p, (const void *const *)tau, none, const_cast<void *>(u), const_cast<void *>(v),
                           const_cast<void *>(w), stats, nullptr, nullptr, 0, 0.0, c);
        p.partials = (float *)partials;
        p.ticket = ticket;
        if (h->vel_dtype == WMIBM_BF16)
            k_wall<float, __nv_bfloat16><<<blocks, 256, 0, stream>>>(p);
        else
            k_wall<float, float><<<blocks, 256, 0, stream>>>(p);
    }
    return cuda_status(h, cudaGetLastError(), "k_wall launch");
}

// The wall model at every band node and the solid zeros (persistent kernel).
int wall_model(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
               wmibm_band_stats *stats, const void *logz0, cudaStream_t stream)
{
    if (stats && h->nrec == 0) {
        cudaError_t e = cudaMemsetAsync(stats, 0, 2 * sizeof(wmibm_band_stats), stream);
        if (e != cudaSuccess) return cuda_status(h, e, "clear stats");
        stats = nullptr;
    }
    if (h->dtype == WMIBM_F64) return launch_wall<double, double>(h, tau, u, v, w, stats, logz0, stream);
    if (h->vel_dtype == WMIBM_BF16)
        return launch_wall<float, __nv_bfloat16>(h, tau, u, v, w, stats, logz0, stream);
    return launch_wall<float, float>(h, tau, u, v, w, stats, logz0, stream);
}

}  // namespace wmibm
