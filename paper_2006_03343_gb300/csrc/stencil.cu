// Bulk-copy (TMA) pipelined stencil for f = -div(tau) (Eq. 2, Eq. 18, Eqs. 15-16
// of Liu & Stevens, arXiv:2006.03343), the persistent wall-model kernel
// (Sec. 3.3), and the body mask (Eq. 27), for one terrain or for a batch of
// terrains ("members") of uneven grid sizes in the same launches.
//
// Stencil: every member's grid is cut into strips of TY full x-rows
// (j0 .. j0+TY-1); the (member, strip, level) units are split evenly over a
// persistent grid.  Per block, lane 0 of warp 0 is the producer: it issues 1D
// bulk copies of the rows a stage needs into a ring of S shared-memory stages
// and arms the stage's "full" mbarrier with the byte count.  A stage at level k
// has two halves in two rings of shared-memory slots:
//   half A: txx at k (TY rows), txy, tyy at k (TY + 2 rows: y-halo)
//   half B: tzz at k (TY rows), txz at k+1 (TY rows), tyz at k+1 (TY + 2 rows)
// and the half B of the stage before it supplies txz, tyz at k and tzz at k-1,
// so every stress row is fetched from HBM once per strip.  Half A is released
// as soon as its stage is consumed, half B after the next stage: the ring of
// half B has one slot more, and the producer runs (stages - 1) stages ahead.  A segment (consecutive
// levels of one strip of one member) starts with a prologue stage that holds
// only tzz at k-1 and txz, tyz at k.  Consumer warps form f for the TY rows,
// with x-neighbours from warp shuffles and periodic wrap inside the staged full
// rows, and release the stage through the "empty" mbarrier.
//
// Units are split into "clean" ones, whose stage rows hold no band or solid
// node, and "dirty" ones; each block streams its share of clean units first.
// The step runs the wall kernel, then the stencil kernel as its programmatic
// dependent: before its first dirty stage, and before the body mask (which may
// change the velocity only after every band stencil has read it), the stencil
// kernel waits on the grid dependency.
//
// Wall kernel: the threads of the grid share the band records (two per thread
// and round, every independent load issued before the stores) and the solid
// runs (a warp zeroes one run at a time with coalesced stores).
//
// Every mbarrier wait is bounded: on time-out the kernel records a status code
// in device memory and leaves its loops.
#include <algorithm>

#include "band.cuh"
#include "members.cuh"
#include "tma.cuh"

using namespace wmibm;

namespace {

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    static constexpr int V = 4;
};
template <>
struct VecOf<double> {
    static constexpr int V = 2;
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

// Views of a member's fields for the producer and the consumers (filled with
// constant-offset loads, so that nothing is copied to local memory).
template <typename T>
struct ProdView {
    const T *tau[6];
    int32_t nx, ny, nz, ty;
};

template <typename T>
struct ConsView {
    T *f[3];
    int32_t nx, ny, nz, ty;
    T cx, cy, cz;
    // this lane's first (row, vector column) of a stage and the step between
    // its groups (ncons * 32 groups = dr rows + dq columns), per member
    int32_t nq, r0, q0, dr, dq;
};

template <typename T>
__device__ __forceinline__ void load_prod(const KParams<T> &p, int m, ProdView<T> &v)
{
    if (p.nmembers == 1) {
        v.tau[0] = p.one.tau[0]; v.tau[1] = p.one.tau[1]; v.tau[2] = p.one.tau[2];
        v.tau[3] = p.one.tau[3]; v.tau[4] = p.one.tau[4]; v.tau[5] = p.one.tau[5];
        v.nx = p.one.nx; v.ny = p.one.ny; v.nz = p.one.nz; v.ty = p.one.rows;
    } else {
        const Member<T> *mm = p.list + m;
        v.tau[0] = mm->tau[0]; v.tau[1] = mm->tau[1]; v.tau[2] = mm->tau[2];
        v.tau[3] = mm->tau[3]; v.tau[4] = mm->tau[4]; v.tau[5] = mm->tau[5];
        v.nx = mm->nx; v.ny = mm->ny; v.nz = mm->nz; v.ty = mm->rows;
    }
}

template <typename T>
__device__ __forceinline__ void load_cons(const KParams<T> &p, int m, ConsView<T> &v)
{
    if (p.nmembers == 1) {
        v.f[0] = p.one.f[0]; v.f[1] = p.one.f[1]; v.f[2] = p.one.f[2];
        v.nx = p.one.nx; v.ny = p.one.ny; v.nz = p.one.nz; v.ty = p.one.rows;
        v.cx = p.one.cx; v.cy = p.one.cy; v.cz = p.one.cz;
    } else {
        const Member<T> *mm = p.list + m;
        v.f[0] = mm->f[0]; v.f[1] = mm->f[1]; v.f[2] = mm->f[2];
        v.nx = mm->nx; v.ny = mm->ny; v.nz = mm->nz; v.ty = mm->rows;
        v.cx = mm->cx; v.cy = mm->cy; v.cz = mm->cz;
    }
}

// Unit-space shape of member m.
struct MemberUnits {
    int32_t nstrips, nz, da, db;
    int64_t c_off, d_off;
};

template <typename T>
__device__ __forceinline__ MemberUnits load_units(const KParams<T> &p, int m)
{
    MemberUnits u;
    if (p.nmembers == 1) {
        u.nstrips = p.one.nstrips; u.nz = p.one.nz; u.da = p.one.da; u.db = p.one.db;
        u.c_off = 0; u.d_off = 0;
    } else {
        const Member<T> *mm = p.list + m;
        u.nstrips = mm->nstrips; u.nz = mm->nz; u.da = mm->da; u.db = mm->db;
        u.c_off = mm->c_off; u.d_off = mm->d_off;
    }
    return u;
}

// Member holding index i of the clean (phase 0) or dirty (phase 1) unit space.
template <typename T>
__device__ int find_member(const KParams<T> &p, int phase, int64_t i)
{
    if (p.nmembers == 1) return 0;
    int lo = 0, hi = p.nmembers - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t off = phase == 0 ? p.list[mid].c_off : p.list[mid].d_off;
        if (off <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Member holding index g of a concatenated per-member space (batch): the last
// member whose first index (the Member field `first`) is <= g.
template <typename T>
__device__ int find_member_at(const KParams<T> &p, int64_t Member<T>::*first, int64_t g)
{
    int lo = 0, hi = p.nmembers - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.list[mid].*first <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Sequence of stages a block processes: its share of the clean units, then its
// share of the dirty units, cut into segments of consecutive levels of one
// strip of one member; each segment starts with a prologue stage followed by
// one main stage per level.
//
// Interleaved form (one launch, wall model inside): the block also owns a
// share of "wall items", slices of wall_chunk consecutive records of the
// concatenated band-record space.  Each is one stage (the producer stages the
// records, the consumers evaluate them); they are spread over the first half
// of the block's clean units, between units, and any left go before the first
// dirty unit.  After a wall stage the pending unit restarts with a prologue.
// A block always has at least one wall stage (with no records when the item
// space is smaller than the grid): its first zeroes the block's share of the
// solid runs, its last counts the block into wall_done.
template <typename T>
struct StageIter {
    const KParams<T> *pp;
    int64_t c1, d0, d1;           // block ranges (clean [c0, c1), dirty [d0, d1))
    int64_t idx;                  // global index in the current phase's space
    int phase;                    // 0 clean, 1 dirty, 2 done
    int m;                        // member
    MemberUnits mu;
    int32_t s, k;
    bool prologue, done, dirty, new_member;
    // interleaved form
    bool inter, wall, sdone;      // wall: the current stage is a wall stage; sdone: no unit left
    bool dyn;                     // units taken in runs from the launch's counters (producer only)
    int64_t wf, wn, wj, wrec;     // first wall item, wall stages, next wall stage, items with records
    int64_t nclean, cdone;        // the block's clean units, clean main stages emitted

    // a wall stage is due before the pending unit
    __device__ __forceinline__ bool wall_due() const
    {
        if (!inter || wj >= wn) return false;
        if (sdone || phase != 0) return true;
        return cdone >= (wj * nclean) / (2 * wn);
    }
    // record range [a, e) of the current wall stage (empty for a block without record items)
    __device__ __forceinline__ void wall_range(int64_t &a, int64_t &e) const
    {
        if (wj >= wrec) {
            a = e = 0;
            return;
        }
        const int64_t q = (int64_t)pp->wall_chunk;
        a = (wf + wj) * q;
        e = min(a + q, pp->rec_total);
    }

    __device__ void locate()
    {
        int m2 = m;
        if (m < 0 || idx < (phase == 0 ? mu.c_off : mu.d_off) ||
            idx >= (phase == 0 ? mu.c_off + (int64_t)mu.nstrips * (mu.da + (mu.nz - mu.db))
                               : mu.d_off + (int64_t)mu.nstrips * (mu.db - mu.da)))
            m2 = find_member(*pp, phase, idx);
        if (m2 != m) {
            m = m2;
            mu = load_units(*pp, m);
            new_member = true;
        }
        // member-local unit index (fits 32 bits: a member has < 2^31 units)
        const uint32_t li = (uint32_t)(idx - (phase == 0 ? mu.c_off : mu.d_off));
        if (phase == 0) {
            const uint32_t lc = (uint32_t)(mu.da + (mu.nz - mu.db));
            s = (int32_t)(li / lc);
            const int32_t r = (int32_t)(li - (uint32_t)s * lc);
            k = r < mu.da ? r : mu.db + (r - mu.da);
        } else {
            const uint32_t ld = (uint32_t)(mu.db - mu.da);
            s = (int32_t)(li / ld);
            k = mu.da + (int32_t)(li - (uint32_t)s * ld);
        }
    }
    __device__ void settle()
    {
        if (dyn) {
            // take the next run of units of the current phase (guided: a share of
            // what is left, at least dyn_chunk units, so that the runs are long while
            // much is left and short towards the end); when the phase's counter has
            // passed its total, move on to the dirty units, then stop
            while (phase < 2 && idx >= (phase == 0 ? c1 : d1)) {
                const int64_t total = phase == 0 ? pp->clean_total : pp->dirty_total;
                unsigned long long *ctr = pp->dyn_ctr + phase;
                const int64_t seen = (int64_t)*(volatile unsigned long long *)ctr;
                int64_t take = (total - seen) / (2 * (int64_t)gridDim.x);
                if (take < pp->dyn_chunk) take = pp->dyn_chunk;
                const int64_t lo = (int64_t)atomicAdd(ctr, (unsigned long long)take);
                if (lo < total) {
                    idx = lo;
                    const int64_t hi = min(total, lo + take);
                    if (phase == 0)
                        c1 = hi;
                    else
                        d1 = hi;
                } else {
                    ++phase;
                    idx = 0;
                    d1 = 0;
                }
            }
        } else {
            while (phase < 2 && idx >= (phase == 0 ? c1 : d1)) {
                ++phase;
                idx = d0;
            }
        }
        sdone = phase >= 2;
        if (!sdone) {
            locate();
            prologue = true;
            dirty = phase == 1;
        }
    }
    // after the stage sequence moved on: a wall stage may be due before the pending unit
    __device__ __forceinline__ void pick()
    {
        wall = wall_due();
        done = sdone && !wall;
    }
    __device__ void init(const KParams<T> &p)
    {
        pp = &p;
        // the stencil blocks of the launch (dedicated wall blocks come first)
        const int64_t wb = p.wall_blocks > 0 ? p.wall_blocks : 0;
        const int64_t sb = blockIdx.x - wb, nsb = gridDim.x - wb;
        const int64_t C = p.clean_total, D = p.dirty_total;
        const int64_t c0 = C * sb / nsb;
        c1 = C * (sb + 1) / nsb;
        d0 = D * sb / nsb;
        d1 = D * (sb + 1) / nsb;
        m = -1;
        phase = 0;
        idx = c0;
        new_member = false;
        dyn = p.dyn_chunk > 0;
        if (dyn) {
            idx = c1 = d0 = d1 = 0;
        }
        inter = p.interleave != 0;
        nclean = c1 - c0;
        cdone = 0;
        wj = 0;
        if (inter) {
            const int64_t NW = p.wall_items;
            wf = NW * sb / nsb;
            wrec = NW * (sb + 1) / nsb - wf;
            wn = wrec > 0 ? wrec : 1;
        } else {
            wf = wn = wrec = 0;
        }
        settle();
        pick();
    }
    // Next stage: the prologue's main stage, or the next unit in the member's
    // order (clean: levels 0 .. da-1 then db .. nz-1 of a strip; dirty: da ..
    // db-1), found without a division; a unit that does not continue the level
    // sequence of the same strip starts a new segment.  In the interleaved form
    // a due wall stage comes first.
    __device__ void next()
    {
        new_member = false;
        if (wall) {
            // back to the pending unit, which restarts its segment
            ++wj;
            if (!sdone) prologue = true;
            pick();
            return;
        }
        if (prologue) {
            prologue = false;
            return;
        }
        if (!dirty) ++cdone;
        advance();
        pick();
    }
    __device__ void advance()
    {
        ++idx;
        if (idx >= (phase == 0 ? c1 : d1)) {
            settle();
            return;
        }
        const int32_t k0 = k;
        int32_t kn = k + 1;
        if (phase == 0) {
            if (kn == mu.da) kn = mu.db;
            if (kn >= mu.nz) {
                ++s;
                kn = mu.da > 0 ? 0 : mu.db;
            }
        } else if (kn >= mu.db) {
            ++s;
            kn = mu.da;
        }
        k = kn;
        if (s >= mu.nstrips) {
            locate();       // the next member with units in this phase
            prologue = true;
            return;
        }
        prologue = k != k0 + 1;
    }
};

// First row of each stress slot in the two halves of a stage of ty-row strips
// (compile-time constants when the row count is a template argument): half A
// holds 3 ty + 4 rows, half B 3 ty + 2.
struct Slots {
    int XX, XY, YY;   // half A
    int ZZ, XZ, YZ;   // half B
    __device__ __forceinline__ explicit Slots(int ty)
        : XX(0), XY(ty), YY(2 * ty + 2), ZZ(0), XZ(ty), YZ(2 * ty) {}
};

// Waits until the preceding kernel of the stream (the wall kernel) has
// completed and its writes are visible (programmatic dependent launch; without
// a programmatic dependency the stream order already guarantees it).
__device__ __forceinline__ void wait_wall_kernel()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch modes of the stencil kernel.
constexpr int kPlain = 0;       // force only: every unit is clean, no dependency
constexpr int kAfterWall = 1;   // programmatic dependent of the wall kernel (dirty units, mask wait on it)
constexpr int kFused = 2;       // the wall phase runs inside the launch (cooperative: all blocks resident)
constexpr int kInterleaved = 3; // the band records are stages of every block's pipeline (cooperative)
constexpr int kWarpSpec = 4;    // wall warps beside the producer and consumers of every block (cooperative)

// Waits until *ctr >= target (acquire at GPU scope).  Gives up after limit_ns,
// recording kDevStatusBarrierTimeout, or as soon as another wait has given up.
__device__ bool wait_counter(const unsigned *ctr, unsigned target, int *status, uint64_t limit_ns)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(64);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((it & 7u) == 0) {
            if (*(volatile int *)status != 0) return false;
            if (global_timer_ns() - t0 > limit_ns) {
                atomicExch(status, kDevStatusBarrierTimeout);
                return false;
            }
        }
    }
}

// Barrier among the consumer warps only (named barrier 1).
__device__ __forceinline__ void consumers_sync(int ncons)
{
    asm volatile("bar.sync 1, %0;" ::"r"(ncons * 32) : "memory");
}

// Blocks that count themselves into wall_done in a single-launch stage.
__device__ __forceinline__ unsigned wall_target(int wall_blocks)
{
    return wall_blocks > 0 ? (unsigned)wall_blocks : gridDim.x;
}

// ------------------------------------------------------------------------- //
// producer: lane 0 of warp 0
// ------------------------------------------------------------------------- //
// Stages the producer of a fused launch issues before its block's wall share is
// done (the rest waits, so that the wall model's gathers meet a quiet memory system).
constexpr uint32_t kStagesBeforeWall = 1;

// Stage header of the dynamic dispensing (producer -> consumers): member, strip,
// level and flags.
constexpr int kHdrPrologue = 1, kHdrNewMember = 2, kHdrDone = 4;

template <typename T, int TY, int MODE>
__device__ void produce(const KParams<T> &p, T *ring_a, T *ring_b, uint64_t *full, uint64_t *empty_a,
                        uint64_t *empty_b, uint64_t *wallbar, int4 *hdr)
{
    const uint32_t SA = (uint32_t)p.stages, SB = SA + 1;
    ProdView<T> v;
    uint32_t g = 0;
    bool released = MODE == kPlain;
    StageIter<T> it;
    for (it.init(p); !it.done; it.next(), ++g) {
        if (it.new_member) load_prod(p, it.m, v);
        if (MODE == kFused && p.wall_blocks == 0 && g == kStagesBeforeWall) {
            if (!mbar_wait(wallbar, 0u, p.status, kDevStatusBarrierTimeout, p.wait_ns)) break;
        }
        const int b = (int)(g % SA), bb = (int)(g % SB);
        if (g >= SA && !mbar_wait(&empty_a[b], ((g / SA) & 1u) ^ 1u, p.status, kDevStatusEmptyTimeout, p.wait_ns)) break;
        if (g >= SB && !mbar_wait(&empty_b[bb], ((g / SB) & 1u) ^ 1u, p.status, kDevStatusEmptyTimeout, p.wait_ns)) break;
        if (MODE == kInterleaved && it.wall) {
            // a wall stage: the item's band records, one bulk copy per member segment
            using Rec = typename RecOf<T>::type;
            int64_t a, e;
            it.wall_range(a, e);
            mbar_arrive_expect_tx(&full[b], (uint32_t)((e - a) * (int64_t)sizeof(Rec)));
            Rec *const dst = reinterpret_cast<Rec *>(ring_a + (size_t)b * p.half_a);
            int wm = (p.nmembers == 1 || e <= a) ? 0 : find_member_at(p, &Member<T>::r_off, a);
            for (int64_t pos = a; pos < e && wm < p.nmembers; ++wm) {
                const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[wm];
                const int64_t end = min(e, mm.r_off + mm.nb_w + mm.nb_uv);
                if (end > pos)
                    bulk_g2s(dst + (pos - a), reinterpret_cast<const Rec *>(mm.rec) + (pos - mm.r_off),
                             (uint32_t)((end - pos) * (int64_t)sizeof(Rec)), &full[b]);
                pos = end;
            }
            continue;
        }
        if (it.dirty && !released) {
            // the stresses written by the wall model must be complete and visible
            // to the bulk copies (async proxy) before a dirty stage
            if (MODE == kAfterWall) {
                wait_wall_kernel();
            } else if (!wait_counter(p.wall_done, wall_target(p.wall_blocks), p.status, p.wait_ns)) {
                break;
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
            released = true;
        }
        if (it.dyn)   // released to the consumers by the arrive below
            hdr[b] = make_int4(it.m, it.s, it.k, (it.prologue ? kHdrPrologue : 0) | (it.new_member ? kHdrNewMember : 0));
        const int32_t nx = v.nx, ny = v.ny;
        const uint32_t row_bytes = (uint32_t)nx * sizeof(T);
        const int64_t plane = (int64_t)nx * ny;
        T *const sta = ring_a + (size_t)b * p.half_a;
        T *const stb = ring_b + (size_t)bb * p.half_b;
        const int ty = TY > 0 ? TY : v.ty;     // rows per strip (template or per member)
        const Slots S_(ty);
        const int32_t j0 = it.s * ty;
        const int32_t k = it.k;
        // rows [jstart, jstart + cnt) of one level (periodic in j) into consecutive
        // slot rows of a half: one bulk copy per contiguous piece (two where the
        // interval wraps)
        auto issue = [&](const T *arr, int32_t lev, int32_t jstart, int32_t cnt, T *half, int32_t slot) {
            const T *base = arr + (int64_t)lev * plane;
            T *dst = half + (size_t)slot * nx;
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
        const T *const txx = v.tau[0], *const txy = v.tau[1], *const tyy = v.tau[2];
        const T *const tzz = v.tau[3], *const txz = v.tau[4], *const tyz = v.tau[5];
        if (it.prologue) {
            const uint32_t rows = (k > 0 ? ty : 0) + ty + (ty + 2);
            mbar_arrive_expect_tx(&full[b], rows * row_bytes);
            if (k > 0) issue(tzz, k - 1, j0, ty, stb, S_.ZZ);
            issue(txz, k, j0, ty, stb, S_.XZ);
            issue(tyz, k, j0 - 1, ty + 2, stb, S_.YZ);
        } else {
            const bool up = k + 1 < v.nz;
            const uint32_t rows = ty + 2 * (ty + 2) + ty + (up ? ty + (ty + 2) : 0);
            mbar_arrive_expect_tx(&full[b], rows * row_bytes);
            issue(txx, k, j0, ty, sta, S_.XX);
            issue(txy, k, j0 - 1, ty + 2, sta, S_.XY);
            issue(tyy, k, j0 - 1, ty + 2, sta, S_.YY);
            issue(tzz, k, j0, ty, stb, S_.ZZ);
            if (up) {
                issue(txz, k + 1, j0, ty, stb, S_.XZ);
                issue(tyz, k + 1, j0 - 1, ty + 2, stb, S_.YZ);
            }
        }
    }
    if (!it.done) {
        // gave up: let the copies already issued land before the block exits
        const uint32_t first = g > SA ? g - SA : 0;
        for (uint32_t q = first; q < g; ++q) mbar_drain(&full[q % SA], (q / SA) & 1u);
    } else if (it.dyn) {
        // one more stage that only tells the consumers there is nothing left
        const int b = (int)(g % SA);
        if (g < SA || mbar_wait(&empty_a[b], ((g / SA) & 1u) ^ 1u, p.status, kDevStatusEmptyTimeout, p.wait_ns)) {
            hdr[b] = make_int4(0, 0, 0, kHdrDone);
            mbar_arrive_expect_tx(&full[b], 0u);
        }
    }
}

// ------------------------------------------------------------------------- //
// consumers: f for the TY rows of a main stage
// ------------------------------------------------------------------------- //
// cur: half A of the stage; curb, prvb: half B of the stage and of the one before.
template <typename T, int TY>
__device__ void consume_level(const ConsView<T> &cv, int ncons, const T *cur, const T *curb, const T *prv,
                              int32_t k, int32_t j0, int cw, int lane)
{
    const int ty = TY > 0 ? TY : cv.ty;         // rows per strip (template or per member)
    const Slots S_(ty);
    constexpr int V = VecOf<T>::V;
    const int32_t nx = cv.nx;
    const int nq = cv.nq;
    const int groups = ty * nq;
    const int64_t plane = (int64_t)nx * cv.ny;
    const bool top = (k == cv.nz - 1);
    const bool bottom = (k == 0);
    const T cx = cv.cx, cy = cv.cy, cz = cv.cz;
    int rl = cv.r0, ql = cv.q0;
    for (int base = cw * 32; base < groups; base += ncons * 32) {
        const int gi = base + lane;
        const bool valid = rl < ty;
        const int r = valid ? rl : ty - 1, q = valid ? ql : nq - 1;
        ql += cv.dq;
        rl += cv.dr;
        if (ql >= nq) {
            ql -= nq;
            ++rl;
        }
        const int i = q * V;
        const int64_t o = (int64_t)k * plane + (int64_t)(j0 + r) * nx + i;
        if (top) {
            Pack<T> z;
            for (int e = 0; e < V; ++e) z.v[e] = T(0);
            if (valid) {
                stg(cv.f[0] + o, z);
                stg(cv.f[1] + o, z);
                stg(cv.f[2] + o, z);
            }
            continue;
        }
        const int im = (i == 0) ? nx - 1 : i - 1;
        const int ip = (i + V == nx) ? 0 : i + V;
        // x-neighbours at the vector edges: from the adjacent lane when it holds
        // the adjacent vector of the same row, else from shared memory
        const bool left_ok = lane > 0 && q > 0;
        const bool right_ok = lane < 31 && q < nq - 1 && gi + 1 < groups;
        auto x_neighbours = [&](const T *row, const Pack<T> &a, T &l, T &rr) {
            l = __shfl_up_sync(0xffffffffu, a.v[V - 1], 1);
            rr = __shfl_down_sync(0xffffffffu, a.v[0], 1);
            if (!left_ok) l = row[im];
            if (!right_ok) rr = row[ip];
        };
        // the three components one after the other, each with only its own
        // operands live (fewer registers, more resident warps)
        {
            const T *XXr = cur + (S_.XX + r) * nx;
            const Pack<T> xx = lds(XXr + i);
            T xxl, xxr;
            x_neighbours(XXr, xx, xxl, xxr);
            const Pack<T> xym = lds(cur + (S_.XY + r) * nx + i), xyp = lds(cur + (S_.XY + r + 2) * nx + i);
            const Pack<T> xz1 = lds(curb + (S_.XZ + r) * nx + i);
            const Pack<T> xz0 = lds(prv + (S_.XZ + r) * nx + i);
            Pack<T> Fx;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const T xxm_ = e == 0 ? xxl : xx.v[e - 1], xxp_ = e == V - 1 ? xxr : xx.v[e + 1];
                Fx.v[e] = -((xxp_ - xxm_) * cx + (xyp.v[e] - xym.v[e]) * cy + (xz1.v[e] - xz0.v[e]) * cz);
            }
            if (valid) stg(cv.f[0] + o, Fx);
        }
        {
            const T *XYc = cur + (S_.XY + r + 1) * nx;
            const Pack<T> xy = lds(XYc + i);
            T xyl, xyr;
            x_neighbours(XYc, xy, xyl, xyr);
            const Pack<T> yym = lds(cur + (S_.YY + r) * nx + i), yyp = lds(cur + (S_.YY + r + 2) * nx + i);
            const Pack<T> yz1 = lds(curb + (S_.YZ + r + 1) * nx + i);
            const Pack<T> yz0 = lds(prv + (S_.YZ + r + 1) * nx + i);
            Pack<T> Fy;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const T xym_ = e == 0 ? xyl : xy.v[e - 1], xyp_ = e == V - 1 ? xyr : xy.v[e + 1];
                Fy.v[e] = -((xyp_ - xym_) * cx + (yyp.v[e] - yym.v[e]) * cy + (yz1.v[e] - yz0.v[e]) * cz);
            }
            if (valid) stg(cv.f[1] + o, Fy);
        }
        {
            const T *XZ0 = prv + (S_.XZ + r) * nx;
            const Pack<T> xz0 = lds(XZ0 + i);
            T xzl, xzr;
            x_neighbours(XZ0, xz0, xzl, xzr);
            const Pack<T> yz0m = lds(prv + (S_.YZ + r) * nx + i), yz0p = lds(prv + (S_.YZ + r + 2) * nx + i);
            const Pack<T> zz = lds(curb + (S_.ZZ + r) * nx + i);
            Pack<T> zzm;
            if (!bottom)
                zzm = lds(prv + (S_.ZZ + r) * nx + i);
            else
                for (int e = 0; e < V; ++e) zzm.v[e] = T(0);
            Pack<T> Fz;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const T xzm_ = e == 0 ? xzl : xz0.v[e - 1], xzp_ = e == V - 1 ? xzr : xz0.v[e + 1];
                const T fz = -((xzp_ - xzm_) * cx + (yz0p.v[e] - yz0m.v[e]) * cy + (zz.v[e] - zzm.v[e]) * cz);
                Fz.v[e] = bottom ? T(0) : fz;
            }
            if (valid) stg(cv.f[2] + o, Fz);
        }
    }
}

template <typename T, typename VEL>
__device__ void wall_phase_fused(const KParams<T> &p, int64_t wb, int64_t nwb, int cw, int nwarps, int lane,
                                 T (*red)[kStatVals]);

template <typename T, typename VEL>
__device__ void wall_stage(const KParams<T> &p, const typename RecOf<T>::type *recs, int64_t a, int64_t e,
                           bool first, bool last, int cw, int lane, unsigned *warps_done);

template <typename T, typename VEL, int TY, int MODE>
__device__ void consume(const KParams<T> &p, const T *ring_a, const T *ring_b, uint64_t *full, uint64_t *empty_a,
                        uint64_t *empty_b, int cw, int lane, T (*red)[kStatVals], uint64_t *wallbar,
                        unsigned *warps_done, const int4 *hdr)
{
    ConsView<T> cv;
    uint32_t g = 0;
    const uint32_t SA = (uint32_t)p.stages, SB = SA + 1;
    // after stage g: its half A is free, and the half B of the stage before it
    auto release = [&](uint32_t gg) {
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&empty_a[gg % SA]);
            if (gg > 0) mbar_arrive(&empty_b[(gg - 1) % SB]);
        }
    };
    if (p.dyn_chunk > 0) {
        // dynamic dispensing: the unit of each stage comes in its header
        for (;; ++g) {
            const int b = (int)(g % SA);
            if (!__all_sync(0xffffffffu, mbar_wait(&full[b], (g / SA) & 1u, p.status, kDevStatusFullTimeout, p.wait_ns)))
                break;
            const volatile int *hv = reinterpret_cast<const volatile int *>(&hdr[b]);
            const int4 hd = make_int4(hv[0], hv[1], hv[2], hv[3]);
            if (hd.w & kHdrDone) break;
            if (hd.w & kHdrNewMember) {
                load_cons(p, hd.x, cv);
                constexpr int V = VecOf<T>::V;
                cv.nq = cv.nx / V;
                const int first = cw * 32 + lane, step = p.ncons * 32;
                cv.r0 = first / cv.nq;
                cv.q0 = first - cv.r0 * cv.nq;
                cv.dr = step / cv.nq;
                cv.dq = step - cv.dr * cv.nq;
            }
            if (!(hd.w & kHdrPrologue))
                consume_level<T, TY>(cv, p.ncons, ring_a + (size_t)b * p.half_a, ring_b + (size_t)(g % SB) * p.half_b,
                                     ring_b + (size_t)((g + SB - 1) % SB) * p.half_b, hd.z,
                                     hd.y * (TY > 0 ? TY : cv.ty), cw, lane);
            release(g);
        }
        return;
    }
    if (MODE == kFused && p.wall_blocks == 0) {
        // the block's wall share first, while the memory system is quiet; then
        // let the producer stream
        wall_phase_fused<T, VEL>(p, blockIdx.x, gridDim.x, cw, p.ncons, lane, red);
        if (cw == 0 && lane == 0) mbar_arrive(wallbar);
    }
    StageIter<T> it;
    for (it.init(p); !it.done; it.next(), ++g) {
        if (it.new_member) {
            load_cons(p, it.m, cv);
            constexpr int V = VecOf<T>::V;
            cv.nq = cv.nx / V;
            const int first = cw * 32 + lane, step = p.ncons * 32;
            cv.r0 = first / cv.nq;
            cv.q0 = first - cv.r0 * cv.nq;
            cv.dr = step / cv.nq;
            cv.dq = step - cv.dr * cv.nq;
        }
        const int b = (int)(g % SA);
        // the whole warp gives up together, so that no lane is left behind at a warp-wide operation
        if (!__all_sync(0xffffffffu, mbar_wait(&full[b], (g / SA) & 1u, p.status, kDevStatusFullTimeout, p.wait_ns)))
            break;
        if (MODE == kInterleaved && it.wall) {
            int64_t a, e;
            it.wall_range(a, e);
            wall_stage<T, VEL>(p, reinterpret_cast<const typename RecOf<T>::type *>(ring_a + (size_t)b * p.half_a),
                               a, e, it.wj == 0, it.wj == it.wn - 1, cw, lane, warps_done);
        } else if (!it.prologue) {
            consume_level<T, TY>(cv, p.ncons, ring_a + (size_t)b * p.half_a, ring_b + (size_t)(g % SB) * p.half_b,
                                 ring_b + (size_t)((g + SB - 1) % SB) * p.half_b, it.k,
                                 it.s * (TY > 0 ? TY : cv.ty), cw, lane);
        }
        release(g);
    }
}

// ------------------------------------------------------------------------- //
// body mask (Eq. 27) over the launch's concatenated body lists
// ------------------------------------------------------------------------- //
// One member's body-mask fields (constant-offset loads into registers).
template <typename T>
struct MaskView {
    void *u, *v, *w;
    const int32_t *body_uv, *body_w;
    int64_t first, n_uv, end;     // member's slice [first, end) of the body space
    const T *gpx, *gpy, *gpz;
    T mask_c;
};

template <typename T>
__device__ __forceinline__ void load_mask(const Member<T> &mm, MaskView<T> &v)
{
    v.u = mm.u; v.v = mm.v; v.w = mm.w;
    v.body_uv = mm.body_uv; v.body_w = mm.body_w;
    v.first = mm.body_off;
    v.n_uv = mm.nbody_uv;
    v.end = mm.body_off + mm.nbody_uv + mm.nbody_w;
    v.gpx = mm.gpx; v.gpy = mm.gpy; v.gpz = mm.gpz;
    v.mask_c = mm.mask_c;
}

// Eq. 27 over the launch's concatenated body lists (uv-body nodes of a member
// first, then its w-body nodes): thread tid takes indices tid, tid + stride, ...
template <typename T, typename VEL>
__device__ void mask_phase(const KParams<T> &p, int64_t tid, int64_t stride)
{
    const int64_t total = p.body_total;
    if (tid >= total) return;
    int m = p.nmembers == 1 ? 0 : find_member_at(p, &Member<T>::body_off, tid);
    MaskView<T> mv;
    load_mask(p.nmembers == 1 ? p.one : p.list[m], mv);
    for (int64_t t = tid; t < total; t += stride) {
        while (t >= mv.end) load_mask(p.list[++m], mv);
        const int64_t lt = t - mv.first;
        if (lt < mv.n_uv) {
            const int32_t idx = __ldg(mv.body_uv + lt);
            reinterpret_cast<VEL *>(mv.u)[idx] = to_vel<VEL, T>(mv.gpx ? mv.mask_c * __ldg(mv.gpx + idx) : T(0));
            reinterpret_cast<VEL *>(mv.v)[idx] = to_vel<VEL, T>(mv.gpy ? mv.mask_c * __ldg(mv.gpy + idx) : T(0));
        } else {
            const int32_t idx = __ldg(mv.body_w + (lt - mv.n_uv));
            reinterpret_cast<VEL *>(mv.w)[idx] = to_vel<VEL, T>(mv.gpz ? mv.mask_c * __ldg(mv.gpz + idx) : T(0));
        }
    }
}

// ------------------------------------------------------------------------- //
// wall kernels
// ------------------------------------------------------------------------- //
template <typename T, typename VEL>
__device__ __forceinline__ BandOut<T> band_of(const Member<T> &mm, int64_t t)
{
    return band_model<T, VEL>(mm.rec, t, t < mm.nb_w, reinterpret_cast<const VEL *>(mm.u),
                              reinterpret_cast<const VEL *>(mm.v), reinterpret_cast<const VEL *>(mm.w), mm.nx, mm.ny,
                              (int64_t)mm.nx * mm.ny, mm.logz0, mm.log_phi_c, mm.kappa2);
}

template <typename T>
__device__ __forceinline__ void store_band(const Member<T> &mm, const BandOut<T> &o, bool is_w)
{
    if (is_w) {
        const_cast<T *>(mm.tau[4])[o.idx] = o.t0;
        const_cast<T *>(mm.tau[5])[o.idx] = o.t1;
    } else {
        const_cast<T *>(mm.tau[0])[o.idx] = o.t0;
        const_cast<T *>(mm.tau[1])[o.idx] = o.t1;
        const_cast<T *>(mm.tau[2])[o.idx] = o.t2;
        const_cast<T *>(mm.tau[3])[o.idx] = o.t3;
    }
}

// Descriptor of solid run t of one member (w-runs first), or an empty run past the end.
template <typename T>
__device__ __forceinline__ int2 run_at(const Member<T> &mm, int64_t t)
{
    return t < mm.nr_w + mm.nr_uv ? __ldg(t < mm.nr_w ? mm.runs_w + t : mm.runs_uv + (t - mm.nr_w)) : make_int2(0, 0);
}

// Solid runs of one member, warp-cooperative: warp gw of nwarps takes runs
// gw, gw + nwarps, ...: lane q fetches the descriptor of the q-th of them, then
// the warp zeroes them one after the other with coalesced stores.  first: the
// descriptor of this lane's first run, when the caller loaded it early so that
// its latency overlaps other work.
template <typename T>
__device__ void zero_runs(const Member<T> &mm, int64_t gw, int64_t nwarps, int lane, const int2 *first = nullptr)
{
    T *const oxx = const_cast<T *>(mm.tau[0]), *const oxy = const_cast<T *>(mm.tau[1]);
    T *const oyy = const_cast<T *>(mm.tau[2]), *const ozz = const_cast<T *>(mm.tau[3]);
    T *const oxz = const_cast<T *>(mm.tau[4]), *const oyz = const_cast<T *>(mm.tau[5]);
    const int64_t nruns = mm.nr_w + mm.nr_uv;
    for (int64_t base = gw; base < nruns; base += nwarps * 32) {
        const int64_t t = base + (int64_t)lane * nwarps;
        const int2 run = (first && base == gw) ? *first : run_at(mm, t);
        const int nq = (int)min((int64_t)32, (nruns - base + nwarps - 1) / nwarps);
        for (int q = 0; q < nq; ++q) {
            const int32_t start = __shfl_sync(0xffffffffu, run.x, q);
            const int32_t len = __shfl_sync(0xffffffffu, run.y, q);
            const bool is_w = base + (int64_t)q * nwarps < mm.nr_w;
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

// Single terrain: the grid shares the band records two per thread and round;
// band statistics accumulate per thread, are reduced per block and then by the
// last block (into the caller's scratch), or go to the handle's FP64
// accumulator, which the last block out converts when the call asks for the
// statistics (emit_stats) and the stencil launch that follows otherwise.
template <typename T, typename VEL>
__global__ void __launch_bounds__(256) k_wall(KParams<T> p)
{
    __shared__ T red[32][kStatVals];
    __shared__ bool s_last;
    // let the stencil kernel (next in the stream) launch right away
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    T acc[kStatVals];
    stats_identity(acc);
    const Member<T> &mm = p.one;
    const int64_t nrec = mm.nb_w + mm.nb_uv;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    // this lane's first solid-run descriptor, in flight during the band records
    const int2 run0 = run_at(mm, gw + (int64_t)(threadIdx.x & 31) * nwarps);
    for (int64_t t0 = tid; t0 < nrec; t0 += 2 * stride) {
        const int64_t t1 = t0 + stride;
        BandOut<T> a, b;
        a = band_of<T, VEL>(mm, t0);
        if (t1 < nrec) b = band_of<T, VEL>(mm, t1);
        store_band(mm, a, t0 < mm.nb_w);
        stats_add(acc, t0 < mm.nb_w ? 0 : 1, a.tw, a.ur);
        if (t1 < nrec) {
            store_band(mm, b, t1 < mm.nb_w);
            stats_add(acc, t1 < mm.nb_w ? 0 : 1, b.tw, b.ur);
        }
    }
    zero_runs(mm, gw, nwarps, threadIdx.x & 31, &run0);
    if (p.sacc) {
        // statistics into the accumulator
        stats_block_reduce(acc, red);
        if (threadIdx.x == 0) stats_red(acc, p.sacc);
        if (p.emit_stats && threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
            if (s_last) {
                __threadfence();
                stats_emit(p.sacc, p.stats, mm.nb_w, mm.nb_uv, mm.nzc_w, mm.nzc_uv);
                *p.ticket = 0u;
            }
        }
    } else if (p.stats) {
        stats_block_reduce(acc, red);
        stats_finish(acc, red, p.partials, p.ticket, gridDim.x, p.stats, mm.nb_w, mm.nb_uv, mm.nzc_w, mm.nzc_uv);
    }
}

// One member's wall-model fields, held in registers while a thread walks its
// records (constant-offset loads).
template <typename T>
struct WallRegs {
    const void *rec;
    const void *u, *v, *w;
    const Member<T> *src;         // the stress pointers are read from here at store time
    const T *logz0;
    int64_t r_off, nb_w, plane;
    int32_t nx, ny;
    T log_phi_c, kappa2;
};

template <typename T>
__device__ __forceinline__ void load_wall(const Member<T> &mm, WallRegs<T> &r)
{
    r.rec = mm.rec;
    r.u = mm.u; r.v = mm.v; r.w = mm.w;
    r.src = &mm;
    r.logz0 = mm.logz0;
    r.r_off = mm.r_off;
    r.nb_w = mm.nb_w;
    r.nx = mm.nx;
    r.ny = mm.ny;
    r.plane = (int64_t)mm.nx * mm.ny;
    r.log_phi_c = mm.log_phi_c;
    r.kappa2 = mm.kappa2;
}

template <typename T>
__device__ __forceinline__ void store_regs(const WallRegs<T> &r, const BandOut<T> &o, bool is_w)
{
    store_band(*r.src, o, is_w);
}

// A batch's member table in the batch wall kernel's shared memory: per member
// its first band record, record array, first solid run, first uv-run and run
// arrays; roff and runoff end with the totals (nmembers + 1 entries).
struct BatchTable {
    int64_t *roff, *runoff, *uvoff;
    const void **rec;
    const int2 **runs_w, **runs_uv;
};

__device__ __forceinline__ int find_first(const int64_t *first, int n, int64_t g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Solid runs [lo, hi) of the concatenated run space of a batch (runs of member m
// at [run_off, run_off + nr_w + nr_uv), w-runs first), zeroed by one warp: each
// lane loads the descriptors of four batches of 32 consecutive runs at once,
// then the warp zeroes the runs one after the other with coalesced stores.
// Consecutive runs mostly share a member, so the stress pointers are rarely
// reloaded.
template <typename T>
__device__ void zero_runs_range(const KParams<T> &p, const BatchTable &mt, int64_t lo, int64_t hi, int lane)
{
    constexpr int kDepth = 4;
    int cm = -1;
    T *oxx = nullptr, *oxy = nullptr, *oyy = nullptr, *ozz = nullptr, *oxz = nullptr, *oyz = nullptr;
    for (int64_t base = lo; base < hi; base += 32 * kDepth) {
        int2 run[kDepth];
        int mrun[kDepth];
        bool wrun[kDepth];
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int64_t t = base + d * 32 + lane;
            run[d] = make_int2(0, 0);
            mrun[d] = 0;
            wrun[d] = false;
            if (t < hi) {
                const int m = find_first(mt.runoff, p.nmembers, t);
                mrun[d] = m;
                wrun[d] = t < mt.uvoff[m];
                run[d] = __ldg(wrun[d] ? mt.runs_w[m] + (t - mt.runoff[m]) : mt.runs_uv[m] + (t - mt.uvoff[m]));
            }
        }
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int64_t b0 = base + d * 32;
            const int nq = (int)max((int64_t)0, min((int64_t)32, hi - b0));
            for (int q = 0; q < nq; ++q) {
                const int32_t start = __shfl_sync(0xffffffffu, run[d].x, q);
                const int32_t len = __shfl_sync(0xffffffffu, run[d].y, q);
                const int m = __shfl_sync(0xffffffffu, mrun[d], q);
                const bool is_w = __shfl_sync(0xffffffffu, (int)wrun[d], q) != 0;
                if (m != cm) {
                    const Member<T> &mm = p.list[m];
                    oxx = const_cast<T *>(mm.tau[0]); oxy = const_cast<T *>(mm.tau[1]);
                    oyy = const_cast<T *>(mm.tau[2]); ozz = const_cast<T *>(mm.tau[3]);
                    oxz = const_cast<T *>(mm.tau[4]); oyz = const_cast<T *>(mm.tau[5]);
                    cm = m;
                }
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
}

// Batch: a block first copies the member table (record and run offsets and
// arrays) into shared memory, so that no look-up below waits on a chain of
// global loads, and starts the copy of its first chunk of records.  While that
// chunk is on its way, each warp zeroes a contiguous range of the solid runs of
// all members.  Then the block walks its contiguous slice of the concatenated
// band records (so that it meets few members); a thread walks its records in
// increasing order, advancing the member linearly, and accumulates the band
// statistics of the current member in registers.  When its member changes a
// lane adds them to the member's FP64 accumulators in the batch scratch with
// fire-and-forget global reductions; at the end each warp first combines the
// lanes that hold the same member (one reduction per member and warp).  No
// shared-memory FP64 atomics: on this part their compare-and-swap loops run on
// the narrow FP64 pipe and one contended block held the whole grid back.  The
// last block converts the scratch into wmibm_band_stats and clears it for the
// next call.
template <typename T, typename VEL>
__global__ void __launch_bounds__(256, 2) k_wall_batch(KParams<T> p)
{
    __shared__ bool s_last;
    __shared__ uint64_t rbar[2];
    extern __shared__ __align__(128) unsigned char wb_smem[];   // record chunks, then the member table
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    const int64_t R = p.rec_total;
    const int64_t r0 = R * blockIdx.x / gridDim.x, r1 = R * (blockIdx.x + 1) / gridDim.x;
    const bool want_stats = p.stats != nullptr;
    const int nm = p.nmembers;

    T acc[kStatVals];
    stats_identity(acc);
    int nacc = 0;
    auto flush = [&](int mi) {   // this lane's accumulators into member mi's global slots
        stats_red(acc, p.bstats + (int64_t)mi * 8);
        stats_identity(acc);
        nacc = 0;
    };

    // The block's records arrive in shared memory a chunk ahead of use (1D bulk
    // copies, one per member segment of the chunk; two buffers), so that only
    // the velocity gathers remain on each record's latency path.
    using Rec = typename RecOf<T>::type;
    const int bd = blockDim.x;
    const int64_t CH = 2 * (int64_t)bd;                  // records per chunk: two per thread
    const int64_t nchunks = (r1 - r0 + CH - 1) / CH;
    Rec *const rbuf = reinterpret_cast<Rec *>(wb_smem);  // [2][CH]
    // the member table, read from the member list once per block, so that the
    // look-ups below take no dependent global loads
    BatchTable mt;
    mt.roff = reinterpret_cast<int64_t *>(rbuf + 2 * CH);
    mt.runoff = mt.roff + (nm + 1);
    mt.uvoff = mt.runoff + (nm + 1);
    mt.rec = reinterpret_cast<const void **>(mt.uvoff + nm);
    mt.runs_w = reinterpret_cast<const int2 **>(mt.rec + nm);
    mt.runs_uv = mt.runs_w + nm;
    for (int m = threadIdx.x; m <= nm; m += bd) {
        if (m < nm) {
            const Member<T> &mm = p.list[m];
            mt.roff[m] = mm.r_off;
            mt.runoff[m] = mm.run_off;
            mt.uvoff[m] = mm.run_off + mm.nr_w;
            mt.rec[m] = mm.rec;
            mt.runs_w[m] = mm.runs_w;
            mt.runs_uv[m] = mm.runs_uv;
        } else {
            mt.roff[m] = R;
            mt.runoff[m] = p.run_total;
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(&rbar[0], 1);
        mbar_init(&rbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int64_t q) {                        // thread 0: chunk q into buffer q & 1
        const int64_t a = r0 + q * CH, b = min(r1, a + CH);
        Rec *dst = rbuf + (q & 1) * CH;
        mbar_arrive_expect_tx(&rbar[q & 1], (uint32_t)((b - a) * (int64_t)sizeof(Rec)));
        for (int m = find_first(mt.roff, nm, a), pos = 0; pos < b - a && m < nm; ++m) {
            const int64_t end = min(b, mt.roff[m + 1]) - a;
            if (end > pos)
                bulk_g2s(dst + pos, reinterpret_cast<const Rec *>(mt.rec[m]) + (a + pos - mt.roff[m]),
                         (uint32_t)((end - pos) * (int64_t)sizeof(Rec)), &rbar[q & 1]);
            pos = (int)end;
        }
    };
    int64_t issued = 0, consumed = 0;                    // thread 0's bookkeeping
    if (threadIdx.x == 0 && nchunks > 0) {
        issue(0);
        issued = 1;
    }

    // solid runs of every member (a contiguous range per warp), while the first
    // chunk of records is on its way
    {
        const int64_t nwarps = (int64_t)gridDim.x * (bd / 32);
        const int64_t gw = (int64_t)blockIdx.x * (bd / 32) + (threadIdx.x >> 5);
        const int64_t T_ = p.run_total;
        zero_runs_range(p, mt, T_ * gw / nwarps, T_ * (gw + 1) / nwarps, threadIdx.x & 31);
    }

    int cm = r0 < r1 ? find_first(mt.roff, nm, r0) : 0;
    WallRegs<T> M;
    load_wall(p.list[cm], M);
    int64_t r_end = mt.roff[cm + 1];
    for (int64_t q = 0; q < nchunks; ++q) {
        if (threadIdx.x == 0 && q + 1 < nchunks) {       // its buffer was released by the sync below
            issue(q + 1);
            issued = q + 2;
        }
        const bool ok = mbar_wait(&rbar[q & 1], (uint32_t)((q >> 1) & 1), p.status, kDevStatusFullTimeout, p.wait_ns);
        if (ok && threadIdx.x == 0) consumed = q + 1;
        const int64_t c0 = r0 + q * CH, c1 = min(r1, c0 + CH);
        const Rec *const chunk = rbuf + (q & 1) * CH;
        for (int64_t g = c0 + threadIdx.x; ok && g < c1;) {
            if (g >= r_end) {
                if (want_stats && nacc) flush(cm);
                do {
                    ++cm;
                    r_end = mt.roff[cm + 1];
                } while (g >= r_end);
                load_wall(p.list[cm], M);
            }
            const int64_t g1 = g + bd;
            const bool two = g1 < c1 && g1 < r_end;
            const int64_t ta = g - M.r_off, tb = g1 - M.r_off;
            const VEL *const vu = reinterpret_cast<const VEL *>(M.u);
            const VEL *const vv = reinterpret_cast<const VEL *>(M.v);
            const VEL *const vw = reinterpret_cast<const VEL *>(M.w);
            // FP32: both nodes' gathers in flight before any arithmetic; FP64 (twice
            // the registers per value): one node after the other
            constexpr bool kPair = sizeof(T) == 4;
            BandIn<T> ia, ib;
            band_fetch_shared<T, VEL>(chunk + (g - c0), vu, vv, vw, M.nx, M.ny, M.plane, ia);
            if (kPair && two) band_fetch_shared<T, VEL>(chunk + (g1 - c0), vu, vv, vw, M.nx, M.ny, M.plane, ib);
            const BandOut<T> a = band_finish<T>(ia, ta < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
            store_regs(M, a, ta < M.nb_w);
            stats_add(acc, ta < M.nb_w ? 0 : 1, a.tw, a.ur);
            if (two) {
                if (!kPair) band_fetch_shared<T, VEL>(chunk + (g1 - c0), vu, vv, vw, M.nx, M.ny, M.plane, ib);
                const BandOut<T> b = band_finish<T>(ib, tb < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
                store_regs(M, b, tb < M.nb_w);
                stats_add(acc, tb < M.nb_w ? 0 : 1, b.tw, b.ur);
            }
            nacc = 1;
            g += two ? 2 * bd : bd;
        }
        __syncthreads();                                  // buffer q & 1 is free again
    }
    if (threadIdx.x == 0)                                 // after a time-out: let issued copies land
        for (int64_t q = consumed; q < issued; ++q) mbar_drain(&rbar[q & 1], (uint32_t)((q >> 1) & 1));
    if (want_stats) {
        // one warp reduction per member the warp's lanes hold (0 is the identity of
        // every statistic: tau_w <= 0, |U_r| >= 0)
        __syncwarp();
        const int lane = threadIdx.x & 31;
        unsigned pending = __ballot_sync(0xffffffffu, nacc != 0);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const int key = __shfl_sync(0xffffffffu, cm, leader);
            const bool mine = nacc != 0 && cm == key;
            pending &= ~__ballot_sync(0xffffffffu, mine);
            T v[kStatVals];
            for (int s = 0; s < kStatVals; ++s) v[s] = mine ? acc[s] : T(0);
            for (int bnd = 0; bnd < 2; ++bnd) {
                v[4 * bnd + 0] = warp_sum(v[4 * bnd + 0]);
                v[4 * bnd + 1] = warp_sum(v[4 * bnd + 1]);
                v[4 * bnd + 2] = warp_min(v[4 * bnd + 2]);
                v[4 * bnd + 3] = warp_max(v[4 * bnd + 3]);
            }
            if (lane == leader) stats_red(v, p.bstats + (int64_t)key * 8);
        }
    }

    if (!want_stats) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < p.nmembers * 2; q += blockDim.x) {
        const int m = q >> 1, bnd = q & 1;
        double *src = p.bstats + ((int64_t)m * 2 + bnd) * 4;
        wmibm_band_stats st;
        st.count = bnd == 0 ? p.list[m].nb_w : p.list[m].nb_uv;
        st.n_zclamped = bnd == 0 ? p.list[m].nzc_w : p.list[m].nzc_uv;
        st.sum_tw = __ldcg(src + 0);
        st.sum_tw2 = __ldcg(src + 1);
        st.min_tw = -__longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(src + 2)));
        st.max_ur = __longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(src + 3)));
        if (st.min_tw == 0.0) st.min_tw = 0.0;   // no -0 for an empty band
        p.stats[q] = st;
        src[0] = 0.0;
        src[1] = 0.0;
        src[2] = 0.0;
        src[3] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) *p.ticket = 0u;
}

// Solid runs [lo, hi) of the launch's concatenated run space (w-runs of a member
// first), zeroed by warp w of nw: it takes 32 consecutive runs at a time (one
// descriptor per lane), then zeroes them one after the other with coalesced stores.
template <typename T>
__device__ void zero_run_span(const KParams<T> &p, int64_t lo, int64_t hi, int w, int nw, int lane)
{
    int cm = -1;
    T *oxx = nullptr, *oxy = nullptr, *oyy = nullptr, *ozz = nullptr, *oxz = nullptr, *oyz = nullptr;
    for (int64_t base = lo + (int64_t)w * 32; base < hi; base += (int64_t)nw * 32) {
        const int64_t t = base + lane;
        int2 run = make_int2(0, 0);
        int mrun = 0, wrun = 0;
        if (t < hi) {
            mrun = p.nmembers == 1 ? 0 : find_member_at(p, &Member<T>::run_off, t);
            const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[mrun];
            const int64_t lt = t - mm.run_off;
            wrun = lt < mm.nr_w;
            run = __ldg(wrun ? mm.runs_w + lt : mm.runs_uv + (lt - mm.nr_w));
        }
        const int nq = (int)min((int64_t)32, hi - base);
        for (int q = 0; q < nq; ++q) {
            const int32_t start = __shfl_sync(0xffffffffu, run.x, q);
            const int32_t len = __shfl_sync(0xffffffffu, run.y, q);
            const int m = __shfl_sync(0xffffffffu, mrun, q);
            const bool is_w = __shfl_sync(0xffffffffu, wrun, q) != 0;
            if (m != cm) {
                const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[m];
                oxx = const_cast<T *>(mm.tau[0]); oxy = const_cast<T *>(mm.tau[1]);
                oyy = const_cast<T *>(mm.tau[2]); ozz = const_cast<T *>(mm.tau[3]);
                oxz = const_cast<T *>(mm.tau[4]); oyz = const_cast<T *>(mm.tau[5]);
                cm = m;
            }
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

// Wall stage of the interleaved form, run by every consumer warp of the block on
// the records [a, e) of the launch's concatenated band-record space, staged in
// shared memory by the producer: the wall model of Sec. 3.3 at each band node,
// the band statistics of each
// member into its FP64 accumulator (p.bstats: [member][band][sum tau_w, sum
// tau_w^2, bits of -min tau_w, bits of max |U_r|]) with one set of reductions
// per warp and member.  The block's first wall stage also zeroes its share of
// the solid runs.  After its last, every warp makes its stores visible (also to
// the bulk copies of other blocks) and counts itself in a shared counter; the
// warp that completes it counts the block into wall_done.  No block-wide
// barrier is taken here, so a warp that gave up on a bounded wait cannot hold
// the others.
template <typename T, typename VEL>
__device__ void wall_stage(const KParams<T> &p, const typename RecOf<T>::type *recs, int64_t a, int64_t e,
                           bool first, bool last, int cw, int lane, unsigned *warps_done)
{
    const int nct = p.ncons * 32;
    const int tid = cw * 32 + lane;
    const bool want_stats = p.stats != nullptr;
    T acc[kStatVals];
    stats_identity(acc);
    bool nacc = false;
    int cm = -1;
    int64_t r_end = 0;
    WallRegs<T> M;
    for (int64_t g = a + tid; g < e;) {
        if (cm < 0 || g >= r_end) {
            if (want_stats && nacc) {
                stats_red(acc, p.bstats + (int64_t)cm * 8);
                stats_identity(acc);
                nacc = false;
            }
            cm = p.nmembers == 1 ? 0 : find_member_at(p, &Member<T>::r_off, g);
            const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[cm];
            load_wall(mm, M);
            r_end = mm.r_off + mm.nb_w + mm.nb_uv;
        }
        const int64_t g1 = g + nct;
        const bool two = g1 < e && g1 < r_end;
        const int64_t ta = g - M.r_off, tb = g1 - M.r_off;
        const VEL *const vu = reinterpret_cast<const VEL *>(M.u);
        const VEL *const vv = reinterpret_cast<const VEL *>(M.v);
        const VEL *const vw = reinterpret_cast<const VEL *>(M.w);
        // one node's gathers at a time: inside the stencil kernel a second node's 24
        // values in flight would spill the consumers' registers
        constexpr bool kPair = false;
        BandIn<T> ia, ib;
        band_fetch_shared<T, VEL>(recs + (g - a), vu, vv, vw, M.nx, M.ny, M.plane, ia);
        if (kPair && two) band_fetch_shared<T, VEL>(recs + (g1 - a), vu, vv, vw, M.nx, M.ny, M.plane, ib);
        const BandOut<T> oa = band_finish<T>(ia, ta < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
        store_regs(M, oa, ta < M.nb_w);
        stats_add(acc, ta < M.nb_w ? 0 : 1, oa.tw, oa.ur);
        if (two) {
            if (!kPair) band_fetch_shared<T, VEL>(recs + (g1 - a), vu, vv, vw, M.nx, M.ny, M.plane, ib);
            const BandOut<T> ob = band_finish<T>(ib, tb < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
            store_regs(M, ob, tb < M.nb_w);
            stats_add(acc, tb < M.nb_w ? 0 : 1, ob.tw, ob.ur);
        }
        nacc = true;
        g += two ? 2 * nct : nct;
    }
    if (want_stats) {
        const int key = nacc ? cm : -1;
        const unsigned same = __match_any_sync(0xffffffffu, key);
        if (same == 0xffffffffu) {
            if (key >= 0) {
                for (int q = 0; q < 2; ++q) {
                    acc[4 * q + 0] = warp_sum(acc[4 * q + 0]);
                    acc[4 * q + 1] = warp_sum(acc[4 * q + 1]);
                    acc[4 * q + 2] = warp_min(acc[4 * q + 2]);
                    acc[4 * q + 3] = warp_max(acc[4 * q + 3]);
                }
                if (lane == 0) stats_red(acc, p.bstats + (int64_t)key * 8);
            }
        } else if (nacc) {
            stats_red(acc, p.bstats + (int64_t)cm * 8);
        }
    }
    if (first) {
        const int64_t R = p.run_total, G = gridDim.x;
        zero_run_span(p, R * blockIdx.x / G, R * (blockIdx.x + 1) / G, cw, p.ncons, lane);
    }
    if (last) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __threadfence();
        __syncwarp();
        if (lane == 0 && atomicAdd(warps_done, 1u) == (unsigned)p.ncons - 1) {
            __threadfence();
            if (!p.hold_release) atomicAdd(p.wall_done, 1u);
        }
    }
}

// Wall warps of the warp-specialized form: warps ww = 0 .. nww-1 of the block's
// wall group take the block's contiguous slice of the launch's concatenated
// band records (two records' gathers in flight per thread in FP32), then its
// share of the solid runs, while the producer and the consumers of the same
// block stream the clean stencil units.  Band statistics go per member into the
// FP64 accumulators (p.bstats).  When done, every wall warp makes its stores
// visible (also to other blocks' bulk copies) and counts itself in a shared
// counter; the warp that completes it counts the block into wall_done.
template <typename T, typename VEL>
__device__ void wall_warps_run(const KParams<T> &p, int ww, int nww, int lane, unsigned *warps_done)
{
    const int nt = nww * 32;
    const int tid = ww * 32 + lane;
    const int64_t R = p.rec_total, G = gridDim.x, blk = blockIdx.x;
    const int64_t r0 = R * blk / G, r1 = R * (blk + 1) / G;
    const bool want_stats = p.stats != nullptr;
    T acc[kStatVals];
    stats_identity(acc);
    bool nacc = false;
    int cm = -1;
    int64_t r_end = 0;
    WallRegs<T> M;
    for (int64_t g = r0 + tid; g < r1;) {
        if (cm < 0 || g >= r_end) {
            if (want_stats && nacc) {
                stats_red(acc, p.bstats + (int64_t)cm * 8);
                stats_identity(acc);
                nacc = false;
            }
            cm = p.nmembers == 1 ? 0 : find_member_at(p, &Member<T>::r_off, g);
            const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[cm];
            load_wall(mm, M);
            r_end = mm.r_off + mm.nb_w + mm.nb_uv;
        }
        const int64_t g1 = g + nt;
        const bool two = g1 < r1 && g1 < r_end;
        const int64_t ta = g - M.r_off, tb = g1 - M.r_off;
        const VEL *const vu = reinterpret_cast<const VEL *>(M.u);
        const VEL *const vv = reinterpret_cast<const VEL *>(M.v);
        const VEL *const vw = reinterpret_cast<const VEL *>(M.w);
        // FP32: both nodes' gathers in flight before any arithmetic; FP64: one after the other
        constexpr bool kPair = sizeof(T) == 4;
        BandIn<T> ia, ib;
        band_fetch<T, VEL>(M.rec, ta, vu, vv, vw, M.nx, M.ny, M.plane, ia);
        if (kPair && two) band_fetch<T, VEL>(M.rec, tb, vu, vv, vw, M.nx, M.ny, M.plane, ib);
        const BandOut<T> oa = band_finish<T>(ia, ta < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
        store_regs(M, oa, ta < M.nb_w);
        stats_add(acc, ta < M.nb_w ? 0 : 1, oa.tw, oa.ur);
        if (two) {
            if (!kPair) band_fetch<T, VEL>(M.rec, tb, vu, vv, vw, M.nx, M.ny, M.plane, ib);
            const BandOut<T> ob = band_finish<T>(ib, tb < M.nb_w, M.logz0, M.log_phi_c, M.kappa2);
            store_regs(M, ob, tb < M.nb_w);
            stats_add(acc, tb < M.nb_w ? 0 : 1, ob.tw, ob.ur);
        }
        nacc = true;
        g += two ? 2 * nt : nt;
    }
    if (want_stats) {
        const int key = nacc ? cm : -1;
        const unsigned same = __match_any_sync(0xffffffffu, key);
        if (same == 0xffffffffu) {
            if (key >= 0) {
                for (int q = 0; q < 2; ++q) {
                    acc[4 * q + 0] = warp_sum(acc[4 * q + 0]);
                    acc[4 * q + 1] = warp_sum(acc[4 * q + 1]);
                    acc[4 * q + 2] = warp_min(acc[4 * q + 2]);
                    acc[4 * q + 3] = warp_max(acc[4 * q + 3]);
                }
                if (lane == 0) stats_red(acc, p.bstats + (int64_t)key * 8);
            }
        } else if (nacc) {
            stats_red(acc, p.bstats + (int64_t)cm * 8);
        }
    }
    const int64_t RU = p.run_total;
    zero_run_span(p, RU * blk / G, RU * (blk + 1) / G, ww, nww, lane);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    __syncwarp();
    if (lane == 0 && atomicAdd(warps_done, 1u) == (unsigned)nww - 1) {
        __threadfence();
        if (!p.hold_release) atomicAdd(p.wall_done, 1u);
    }
}

// ------------------------------------------------------------------------- //
// stencil kernel
// ------------------------------------------------------------------------- //
// Wall phase of the fused launch, run once by the consumer warps of every block
// at its start; the producer issues only kStagesBeforeWall stages until the
// block is done with it, so the gathers of the wall model meet a quiet memory
// system.  The block's contiguous slice of band records (two per thread and round), its
// share of the solid runs, then the band statistics reduced over the consumer
// warps into the block's partial.  The block then counts itself into wall_done
// (release); the block that completes the count reduces all partials into the
// caller's stats.  Every consumer warp calls this exactly once, so the named
// barriers inside always meet.
template <typename T, typename VEL>
__device__ void wall_phase_fused(const KParams<T> &p, int64_t wb, int64_t nwb, int cw, int nwarps, int lane,
                                 T (*red)[kStatVals])
{
    const Member<T> &mm = p.one;
    const int nct = nwarps * 32;
    const int tid = cw * 32 + lane;
    const int64_t R = mm.nb_w + mm.nb_uv;
    const int64_t r0 = R * wb / nwb, r1 = R * (wb + 1) / nwb;
    T acc[kStatVals];
    stats_identity(acc);
    for (int64_t t0 = r0 + tid; t0 < r1; t0 += 2 * nct) {
        const int64_t t1 = t0 + nct;
        BandOut<T> a, b;
        a = band_of<T, VEL>(mm, t0);
        if (t1 < r1) b = band_of<T, VEL>(mm, t1);
        store_band(mm, a, t0 < mm.nb_w);
        stats_add(acc, t0 < mm.nb_w ? 0 : 1, a.tw, a.ur);
        if (t1 < r1) {
            store_band(mm, b, t1 < mm.nb_w);
            stats_add(acc, t1 < mm.nb_w ? 0 : 1, b.tw, b.ur);
        }
    }
    zero_runs(mm, wb * nwarps + cw, nwb * nwarps, lane);
    // this thread's stress writes: visible at GPU scope and ordered before the
    // async-proxy reads that other blocks issue after acquiring wall_done
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();

    for (int q = 0; q < 2; ++q) {
        acc[4 * q + 0] = warp_sum(acc[4 * q + 0]);
        acc[4 * q + 1] = warp_sum(acc[4 * q + 1]);
        acc[4 * q + 2] = warp_min(acc[4 * q + 2]);
        acc[4 * q + 3] = warp_max(acc[4 * q + 3]);
    }
    if (lane == 0)
        for (int v = 0; v < kStatVals; ++v) red[cw][v] = acc[v];
    consumers_sync(nwarps);
    if (tid == 0) {
        for (int w = 1; w < nwarps; ++w) stats_combine(acc, red[w]);
        if (p.stats) stats_red(acc, p.sacc);     // converted by the last block out of the launch
        __threadfence();
        if (!p.hold_release) atomicAdd(p.wall_done, 1u);
    }
}

template <typename T, typename VEL, int TY, int MODE>
__global__ void __launch_bounds__(512) k_stencil(KParams<T> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T red[16][kStatVals];
    __shared__ uint64_t wallbar; // fused: the block's wall share is done
    __shared__ int s_go;        // consumers: the wall model is complete (mask may run)
    __shared__ unsigned s_wall_warps;   // interleaved: consumer warps done with the block's wall stages
    __shared__ int4 s_hdr[8];           // dynamic dispensing: the unit of each stage
    __shared__ int s_last;      // the block is the last one out of a single-launch stage
    // barriers: full[8] (per half-A slot), empty_a[8], empty_b[9]; then the two rings
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty_a = full + 8;
    uint64_t *empty_b = full + 16;
    T *ring_a = reinterpret_cast<T *>(smem_raw + 256);
    T *ring_b = ring_a + (size_t)p.stages * p.half_a;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < p.stages; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty_a[b], p.ncons);
        }
        for (int b = 0; b <= p.stages; ++b) mbar_init(&empty_b[b], p.ncons);
        mbar_init(&wallbar, 1);
        fence_mbar_init();
        s_wall_warps = 0;
    }
    __syncthreads();

    constexpr int kFirstConsumer = 1;
    if (MODE != kFused && p.emit_stats && blockIdx.x == 0 && threadIdx.x == 0) {
        // statistics of the wall launch before this one (complete: stream order,
        // or the grid dependency of a programmatic launch)
        if (MODE == kAfterWall) wait_wall_kernel();
        stats_emit(p.sacc, p.stats, p.one.nb_w, p.one.nb_uv, p.one.nzc_w, p.one.nzc_uv);
    }
    if (MODE == kFused && p.wall_blocks > 0 && (int)blockIdx.x < p.wall_blocks) {
        // dedicated wall block: every warp evaluates the block's share of the wall model
        wall_phase_fused<T, VEL>(p, blockIdx.x, p.wall_blocks, warp, blockDim.x >> 5, lane, red);
    } else if (warp == 0) {
        // producer: clean stages right away (their rows hold no band or solid
        // entry), dirty stages once the wall model is complete
        if (lane == 0) produce<T, TY, MODE>(p, ring_a, ring_b, full, empty_a, empty_b, &wallbar, s_hdr);
        __syncwarp();
    } else if (MODE == kWarpSpec && warp > p.ncons) {
        // wall warps: the block's slice of the band records and solid runs
        wall_warps_run<T, VEL>(p, warp - 1 - p.ncons, p.wall_warps, lane, &s_wall_warps);
    } else {
        const int cw = warp - kFirstConsumer;
        consume<T, VEL, TY, MODE>(p, ring_a, ring_b, full, empty_a, empty_b, cw, lane, red, &wallbar, &s_wall_warps,
                                  s_hdr);
        if (MODE != kPlain && p.do_mask) {
            // the body mask may change the velocity only after every band stencil read it
            bool go = true;
            if (MODE == kAfterWall) {
                wait_wall_kernel();
            } else {
                consumers_sync(p.ncons);
                if (cw == 0 && lane == 0)
                    s_go = wait_counter(p.wall_done, wall_target(p.wall_blocks), p.status, p.wait_ns) ? 1 : 0;
                consumers_sync(p.ncons);
                go = s_go != 0;
            }
            // over the consumer threads of the stencil blocks (dedicated wall blocks
            // come first and take no part)
            const int nct = p.ncons * 32;
            const int64_t wb = (MODE == kFused && p.wall_blocks > 0) ? p.wall_blocks : 0;
            if (go)
                mask_phase<T, VEL>(p, ((int64_t)blockIdx.x - wb) * nct + (threadIdx.x - 32 * kFirstConsumer),
                                   ((int64_t)gridDim.x - wb) * nct);
        }
    }
    if (MODE == kFused || MODE == kInterleaved || MODE == kWarpSpec) {
        // the last block out converts the band statistics and re-arms both
        // counters for the next launch: every block has passed its waits on
        // wall_done by then
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(p.exit_ticket, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (MODE == kFused) {
                if (threadIdx.x == 0 && p.stats)
                    stats_emit(p.sacc, p.stats, p.one.nb_w, p.one.nb_uv, p.one.nzc_w, p.one.nzc_uv);
            } else if (p.stats) {
                // every member's accumulator [member][band][4] into its two records, then cleared
                for (int q = threadIdx.x; q < 2 * p.nmembers; q += blockDim.x) {
                    const Member<T> &mm = p.nmembers == 1 ? p.one : p.list[q >> 1];
                    double *src = p.bstats + (int64_t)q * 4;
                    wmibm_band_stats st;
                    st.count = (q & 1) ? mm.nb_uv : mm.nb_w;
                    st.n_zclamped = (q & 1) ? mm.nzc_uv : mm.nzc_w;
                    st.sum_tw = __ldcg(src + 0);
                    st.sum_tw2 = __ldcg(src + 1);
                    st.min_tw = -__longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(src + 2)));
                    st.max_ur = __longlong_as_double((long long)__ldcg(reinterpret_cast<unsigned long long *>(src + 3)));
                    if (st.min_tw == 0.0) st.min_tw = 0.0;   // no -0 for an empty band
                    p.stats[q] = st;
                    src[0] = 0.0;
                    src[1] = 0.0;
                    src[2] = 0.0;
                    src[3] = 0.0;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                atomicExch(p.wall_done, 0u);
                if (p.dyn_chunk > 0) {
                    atomicExch(p.dyn_ctr, 0ull);
                    atomicExch(p.dyn_ctr + 1, 0ull);
                }
                atomicExch(p.exit_ticket, 0u);
            }
        }
    } else if (p.dyn_chunk > 0) {
        // the last block out re-arms the dispensing counters for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(p.exit_ticket, 1u) == gridDim.x - 1) {
                __threadfence();
                atomicExch(p.dyn_ctr, 0ull);
                atomicExch(p.dyn_ctr + 1, 0ull);
                atomicExch(p.exit_ticket, 0u);
            }
        }
    }
}

constexpr int kMaxDynSmem = 200 * 1024;

template <typename T, typename VEL, int TY, int MODE>
int launch_stencil_ty(wmibm_handle *h, KParams<T> &p, const StencilConfig &c, cudaStream_t stream, bool pdl,
                      int max_nx)
{
    auto kern = k_stencil<T, VEL, TY, MODE>;
    static bool attr_done = false;      // once per instantiation and process
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return cuda_status(h, e, "stencil smem attribute");
        attr_done = true;
    }
    // TY == 0 (rows per member): the caller sets the halves to the largest member's
    if (TY > 0) {
        p.half_a = (uint32_t)((3 * TY + 4) * max_nx);
        p.half_b = (uint32_t)((3 * TY + 2) * max_nx);
    }
    const size_t smem = 256 + ((size_t)c.stages * p.half_a + (size_t)(c.stages + 1) * p.half_b) * sizeof(T);
    if (smem > (size_t)kMaxDynSmem) return set_error(h, WMIBM_EINVAL, "stencil stages exceed shared memory");
    // dynamic dispensing where the consumers do not walk the stage sequence themselves
    p.dyn_chunk = (MODE == kFused || MODE == kInterleaved) ? 0 : c.dyn_chunk;
    p.dyn_ctr = reinterpret_cast<unsigned long long *>(p.ticket + 4);
    if (MODE == kWarpSpec) {
        p.wall_warps = c.wall_warps > 0 ? c.wall_warps : 3;
        if (1 + p.ncons + p.wall_warps > 16) return set_error(h, WMIBM_EINVAL, "more than 16 warps per block");
    }
    // producer warp + consumer warps (+ wall warps)
    const int threads = 32 * (1 + p.ncons + (MODE == kWarpSpec ? p.wall_warps : 0));
    // occupancy of this shape, cached in the handle
    const int64_t key = (int64_t)MODE | ((int64_t)TY << 4) | ((int64_t)c.stages << 8) |
                        ((int64_t)c.consumer_warps << 12) | ((int64_t)(MODE == kWarpSpec ? p.wall_warps : 0) << 16) |
                        ((int64_t)(TY > 0 ? max_nx : (int)p.half_a) << 20);
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
    const int64_t units = p.clean_total + p.dirty_total;
    int64_t grid = (int64_t)per_sm * h->sm_count;
    if (grid > units) grid = units;
    if (grid < 1) return WMIBM_OK;
    if (MODE == kInterleaved) {
        // wall items: slices of wall_chunk band records, each staged in one stage buffer
        using Rec = typename RecOf<T>::type;
        const int64_t cap = (int64_t)p.half_a * (int64_t)sizeof(T) / (int64_t)sizeof(Rec);
        int64_t q = c.wall_chunk > 0 ? c.wall_chunk : 2 * 32 * (int64_t)p.ncons;
        if (q > cap) q = cap;
        if (q < 1) return set_error(h, WMIBM_EINVAL, "stencil stage holds no band record");
        p.interleave = 1;
        p.wall_chunk = (int)q;
        p.wall_items = (p.rec_total + q - 1) / q;
    }
    if (MODE == kFused && p.wall_blocks < 0) {
        // dedicated wall blocks: one per SM when the grid has at least two blocks
        // per SM, else a quarter of it; the grid grows by them (up to the resident
        // limit) so that the stencil keeps its blocks
        const int64_t resident = (int64_t)per_sm * h->sm_count;
        int64_t wbk = grid >= 2 * (int64_t)h->sm_count ? h->sm_count : std::max<int64_t>(1, grid / 4);
        grid = std::min<int64_t>(grid + wbk, resident);
        if (grid - wbk < 1) wbk = grid - 1;
        p.wall_blocks = wbk > 0 ? (int)wbk : 0;
    }
    if ((MODE == kAfterWall && pdl) || MODE == kFused || MODE == kInterleaved || MODE == kWarpSpec) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        if (MODE == kFused || MODE == kInterleaved || MODE == kWarpSpec) {
            // blocks wait on each other's wall phase: all must be resident
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
        } else {
            // programmatic dependent of the wall kernel launched just before
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
        }
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cuda_status(h, cudaLaunchKernelEx(&cfg, kern, p), "k_stencil launch");
    }
    kern<<<(unsigned)grid, threads, smem, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_stencil launch");
}

template <typename T, typename VEL, int MODE>
int launch_stencil(wmibm_handle *h, KParams<T> &p, const StencilConfig &c, cudaStream_t stream, bool pdl, int max_nx)
{
    switch (c.rows) {
    case 1: return launch_stencil_ty<T, VEL, 1, MODE>(h, p, c, stream, pdl, max_nx);
    case 2: return launch_stencil_ty<T, VEL, 2, MODE>(h, p, c, stream, pdl, max_nx);
    case 4: return launch_stencil_ty<T, VEL, 4, MODE>(h, p, c, stream, pdl, max_nx);
    default: return set_error(h, WMIBM_EINVAL, "stencil rows must be 1, 2 or 4");
    }
}

bool aligned16(const void *q) { return ((uintptr_t)q & 15u) == 0; }

template <typename T>
void single_params(const wmibm_handle *h, KParams<T> &p, bool step)
{
    p.list = nullptr;
    p.nmembers = 1;
    Member<T> &m = p.one;
    if (!step) {
        // plain force: no preceding wall kernel, so every level is clean (the
        // unit decoding in StageIter reads the member's dirty range)
        m.da = 0;
        m.db = 0;
    }
    p.clean_total = (int64_t)m.nstrips * (m.da + (m.nz - m.db));
    p.dirty_total = (int64_t)m.nstrips * (m.db - m.da);
    p.rec_total = m.nb_w + m.nb_uv;
    p.run_total = m.nr_w + m.nr_uv;
    p.body_total = m.nbody_w + m.nbody_uv;
    p.stages = 2;
    p.ncons = 1;
    p.half_a = 0;
    p.half_b = 0;
    p.status = h->dev_status;
    p.do_mask = 0;
    p.partials = (T *)h->partials;
    p.ticket = h->ticket;
    p.stats = nullptr;
    p.bstats = nullptr;
    p.wall_done = h->ticket + 1;
    p.exit_ticket = h->ticket + 2;
    p.sacc = h->sacc;
    p.emit_stats = 0;
    p.wall_blocks = 0;
    p.interleave = 0;
    p.wall_chunk = 0;
    p.wall_items = 0;
    p.wall_warps = 0;
    p.dyn_chunk = 0;
    p.dyn_ctr = nullptr;
    p.wait_ns = h->wait_ns;
    p.hold_release = h->hold_release;
}

template <typename T, typename VEL>
int launch_wall_single(wmibm_handle *h, void *const tau[6], const void *u, const void *v, const void *w,
                       wmibm_band_stats *stats, const void *logz0, void *partials, unsigned *ticket, unsigned blocks,
                       bool emit, cudaStream_t stream)
{
    KParams<T> p;
    fill_member<T>(h, p.one, (const void *const *)tau, nullptr, const_cast<void *>(u), const_cast<void *>(v),
                   const_cast<void *>(w), logz0, nullptr, 0.0, 0);
    single_params<T>(h, p, false);
    p.stats = stats;
    if (partials) {
        // caller scratch: per-block partials and the last-block ticket
        p.partials = (T *)partials;
        p.ticket = ticket;
        p.sacc = nullptr;
    } else if (!stats) {
        p.sacc = nullptr;
    }
    const int wthreads = blocks ? 256 : 32 * (h->tuning.wall_warps > 0 ? h->tuning.wall_warps : 8);
    if (blocks == 0) {
        int wper = 0;
        const int64_t wkey = 0x100000 | wthreads | (sizeof(T) == 8 ? 0x200000 : 0);
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
        if (h->tuning.wall_grid > 0 && h->tuning.wall_grid < wper) wper = h->tuning.wall_grid;
        blocks = (unsigned)std::min<int64_t>((int64_t)wper * h->sm_count, h->partial_blocks);
    }
    // with the accumulator and emit, the wall kernel's last block converts the statistics
    p.emit_stats = (p.sacc && emit) ? 1 : 0;
    k_wall<T, VEL><<<blocks, wthreads, 0, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_wall launch");
}

}  // namespace

namespace wmibm {

// Fills the member descriptor of handle h with the given fields.
template <typename T>
void fill_member(const wmibm_handle *h, Member<T> &m, const void *const tau[6], void *const f[3], void *u, void *v,
                 void *w, const void *logz0, const void *const gradp[3], double dt, int rows)
{
    for (int a = 0; a < 6; ++a) m.tau[a] = (const T *)tau[a];
    for (int a = 0; a < 3; ++a) m.f[a] = f ? (T *)f[a] : nullptr;
    m.u = u; m.v = v; m.w = w;
    m.nx = h->nx; m.ny = h->ny; m.nz = h->nz;
    m.nstrips = rows > 0 ? h->ny / rows : 0;
    m.rows = rows;
    m.cx = (T)(1.0 / (2.0 * h->dx));
    m.cy = (T)(1.0 / (2.0 * h->dy));
    m.cz = (T)(1.0 / h->dz);
    m.da = h->dirty_lo;
    m.db = h->dirty_hi;
    m.c_off = 0; m.d_off = 0;
    m.rec = h->rec;
    m.nb_w = h->lists.n[WMIBM_LIST_BAND_W];
    m.nb_uv = h->lists.n[WMIBM_LIST_BAND_UV];
    m.nzc_w = h->nzclamp[0];
    m.nzc_uv = h->nzclamp[1];
    m.r_off = 0;
    m.runs_w = h->runs[0]; m.runs_uv = h->runs[1];
    m.nr_w = h->nruns[0]; m.nr_uv = h->nruns[1];
    m.run_off = 0;
    m.body_w = h->lists.p[WMIBM_LIST_BODY_W];
    m.body_uv = h->lists.p[WMIBM_LIST_BODY_UV];
    m.nbody_w = h->lists.n[WMIBM_LIST_BODY_W];
    m.nbody_uv = h->lists.n[WMIBM_LIST_BODY_UV];
    m.body_off = 0;
    m.gpx = gradp ? (const T *)gradp[0] : nullptr;
    m.gpy = gradp ? (const T *)gradp[1] : nullptr;
    m.gpz = gradp ? (const T *)gradp[2] : nullptr;
    m.mask_c = (T)(1.5 * dt);
    m.logz0 = (const T *)logz0;
    m.log_phi_c = (T)log(h->phi_c);
    m.kappa2 = (T)(h->kappa * h->kappa);
}

template void fill_member<float>(const wmibm_handle *, Member<float> &, const void *const[6], void *const[3], void *,
                                 void *, void *, const void *, const void *const[3], double, int);
template void fill_member<double>(const wmibm_handle *, Member<double> &, const void *const[6], void *const[3],
                                  void *, void *, void *, const void *, const void *const[3], double, int);

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
    // shared memory of the two rings: `stages` half-A slots of 3 ty + 4 rows of nx
    // elements and stages + 1 half-B slots of 3 ty + 2 rows
    auto ring_bytes = [&](int rows, int stages) {
        return ((size_t)stages * (3 * rows + 4) + (size_t)(stages + 1) * (3 * rows + 2)) * h->nx * es;
    };
    c.rows = h->tuning.rows;
    c.stages = h->tuning.stages;
    const bool default_shape = c.rows == 0 && c.stages == 0 && h->tuning.consumer_warps == 0;
    if (c.rows == 0) {
        // default: the shape the autotuner keeps for the measured grids (nx 256 and
        // 512): 4-row strips and two stages; narrower strips where the rows do not
        // divide ny or the rings would not fit
        c.rows = 4;
        while (c.rows > 1 && (h->ny % c.rows != 0 || h->ny < c.rows + 2 ||
                              ring_bytes(c.rows, c.stages > 0 ? c.stages : 2) + 256 > (size_t)kMaxDynSmem))
            c.rows /= 2;
    }
    if (!(c.rows == 1 || c.rows == 2 || c.rows == 4)) return false;
    if (h->ny % c.rows != 0 || h->ny < c.rows + 2) return false;
    if (c.stages == 0) c.stages = 2;
    if (c.stages < 2 || c.stages > 8) return false;
    if (ring_bytes(c.rows, c.stages) + 256 > (size_t)kMaxDynSmem) return false;
    // default consumers: 4, or 8 when the rings leave room for one block per SM only
    c.consumer_warps = h->tuning.consumer_warps > 0
                           ? h->tuning.consumer_warps
                           : (default_shape && ring_bytes(c.rows, c.stages) + 256 > 113 * 1024 ? 8 : 4);
    c.wall_warps = h->tuning.wall_warps;
    if (1 + c.consumer_warps > 16) return false;
    c.blocks_per_sm = h->tuning.blocks_per_sm;
    c.wall_chunk = h->tuning.wall_chunk;
    c.dyn_chunk = h->tuning.dyn_chunk;
    c.wall_grid = h->tuning.wall_grid;
    *out = c;
    return true;
}

// emit: NULL, or the stats of the wall launch just before, converted by block 0.
int stencil_force(wmibm_handle *h, const void *const tau[6], void *const f[3], const StencilConfig &c,
                  cudaStream_t stream, wmibm_band_stats *emit)
{
    if (h->dtype == WMIBM_F64) {
        KParams<double> p;
        fill_member<double>(h, p.one, tau, f, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, c.rows);
        single_params<double>(h, p, false);
        p.stages = c.stages;
        p.ncons = c.consumer_warps;
        p.stats = emit;
        p.emit_stats = emit != nullptr;
        return launch_stencil<double, double, kPlain>(h, p, c, stream, false, h->nx);
    }
    KParams<float> p;
    fill_member<float>(h, p.one, tau, f, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, c.rows);
    single_params<float>(h, p, false);
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    p.stats = emit;
    p.emit_stats = emit != nullptr;
    return launch_stencil<float, float, kPlain>(h, p, c, stream, false, h->nx);
}

// The pipelined stencil followed, in the same launch, by the body mask (Eq. 27).
// With pdl the launch is a programmatic dependent of the preceding kernel.
int stencil_force_mask(wmibm_handle *h, void *u, void *v, void *w, const void *const tau[6], void *const f[3],
                       const void *const gradp[3], double dt, const StencilConfig &c, bool pdl, cudaStream_t stream,
                       wmibm_band_stats *emit)
{
    if (h->dtype == WMIBM_F64) {
        KParams<double> p;
        fill_member<double>(h, p.one, tau, f, u, v, w, nullptr, gradp, dt, c.rows);
        single_params<double>(h, p, true);
        p.stages = c.stages;
        p.ncons = c.consumer_warps;
        p.do_mask = 1;
        p.stats = emit;
        p.emit_stats = emit != nullptr;
        return launch_stencil<double, double, kAfterWall>(h, p, c, stream, pdl, h->nx);
    }
    KParams<float> p;
    fill_member<float>(h, p.one, tau, f, u, v, w, nullptr, gradp, dt, c.rows);
    single_params<float>(h, p, true);
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    p.do_mask = 1;
    p.stats = emit;
    p.emit_stats = emit != nullptr;
    if (h->vel_dtype == WMIBM_BF16)
        return launch_stencil<float, __nv_bfloat16, kAfterWall>(h, p, c, stream, pdl, h->nx);
    return launch_stencil<float, float, kAfterWall>(h, p, c, stream, pdl, h->nx);
}

template <typename T, typename VEL>
int step_fused_impl(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *const f[3],
                    const void *const gradp[3], double dt, int do_mask, wmibm_band_stats *stats,
                    const StencilConfig &c, bool dedicated, cudaStream_t stream)
{
    KParams<T> p;
    fill_member<T>(h, p.one, (const void *const *)tau, f, u, v, w, h->logz0, gradp, dt, c.rows);
    single_params<T>(h, p, true);
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    p.do_mask = do_mask;
    p.stats = stats;
    p.wall_blocks = dedicated ? -1 : 0;
    return launch_stencil<T, VEL, kFused>(h, p, c, stream, false, h->nx);
}

// The whole stage in one cooperative launch with the band records cut into
// wall items that are stages of every block's pipeline, between its clean units.
// warp_spec: the wall model in wall warps beside the producer and consumers instead.
template <typename T, typename VEL>
int step_interleaved_impl(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *const f[3],
                          const void *const gradp[3], double dt, int do_mask, wmibm_band_stats *stats,
                          const StencilConfig &c, bool warp_spec, cudaStream_t stream)
{
    KParams<T> p;
    fill_member<T>(h, p.one, (const void *const *)tau, f, u, v, w, h->logz0, gradp, dt, c.rows);
    single_params<T>(h, p, true);
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    p.do_mask = do_mask;
    p.stats = stats;
    p.bstats = h->sacc;           // one member: the accumulator has the [band][4] layout
    if (warp_spec) return launch_stencil<T, VEL, kWarpSpec>(h, p, c, stream, false, h->nx);
    return launch_stencil<T, VEL, kInterleaved>(h, p, c, stream, false, h->nx);
}

// The whole stage in one cooperative launch: the wall model (Sec. 3.3) by the
// consumer warps of every block while the producers stream the clean stages,
// the forcing (Eq. 18) once the wall model is complete where a stage needs it,
// and with do_mask the body mask (Eq. 27).  force_path 5: the wall model as
// interleaved stages of every block's pipeline instead.
int stencil_step_fused(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *const f[3],
                       const void *const gradp[3], double dt, int do_mask, wmibm_band_stats *stats,
                       const StencilConfig &c, cudaStream_t stream)
{
    if (h->tuning.force_path == 5 || h->tuning.force_path == 6) {
        const bool ws = h->tuning.force_path == 6;
        if (h->dtype == WMIBM_F64)
            return step_interleaved_impl<double, double>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, ws,
                                                         stream);
        if (h->vel_dtype == WMIBM_BF16)
            return step_interleaved_impl<float, __nv_bfloat16>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, ws,
                                                                stream);
        return step_interleaved_impl<float, float>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, ws, stream);
    }
    const bool dedicated = h->tuning.force_path == 4;   // dedicated wall blocks
    if (h->dtype == WMIBM_F64)
        return step_fused_impl<double, double>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, dedicated,
                                               stream);
    if (h->vel_dtype == WMIBM_BF16)
        return step_fused_impl<float, __nv_bfloat16>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, dedicated,
                                                     stream);
    return step_fused_impl<float, float>(h, u, v, w, tau, f, gradp, dt, do_mask, stats, c, dedicated, stream);
}

// The wall model at every band node and the solid zeros (persistent kernel).
// emit: convert the statistics here (the wall kernel's last block); false when
// the stencil launch that follows converts them.
int wall_model(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
               wmibm_band_stats *stats, const void *logz0, cudaStream_t stream, bool emit)
{
    if (h->dtype == WMIBM_F64)
        return launch_wall_single<double, double>(h, tau, u, v, w, stats, logz0, nullptr, nullptr, 0, emit, stream);
    if (h->vel_dtype == WMIBM_BF16)
        return launch_wall_single<float, __nv_bfloat16>(h, tau, u, v, w, stats, logz0, nullptr, nullptr, 0, emit,
                                                        stream);
    return launch_wall_single<float, float>(h, tau, u, v, w, stats, logz0, nullptr, nullptr, 0, emit, stream);
}

// The wall kernel with caller-provided reduction scratch and grid size (used by
// the entry point whose scratch lives in a static device array).
int wall_model_with_scratch(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                            wmibm_band_stats *stats, void *partials, unsigned *ticket, unsigned blocks,
                            cudaStream_t stream)
{
    if (h->dtype == WMIBM_F64)
        return launch_wall_single<double, double>(h, tau, u, v, w, stats, h->logz0, partials, ticket, blocks, true,
                                                  stream);
    if (h->vel_dtype == WMIBM_BF16)
        return launch_wall_single<float, __nv_bfloat16>(h, tau, u, v, w, stats, h->logz0, partials, ticket, blocks,
                                                        true, stream);
    return launch_wall_single<float, float>(h, tau, u, v, w, stats, h->logz0, partials, ticket, blocks, true,
                                            stream);
}

// One batched step: the batch wall kernel, then the batch stencil (force + mask)
// as its programmatic dependent (form 3); or one cooperative launch of the batch
// stencil with every member's band records as wall stages of its blocks (form 5)
// or in wall warps beside its producer and consumers (form 6).
// tmpl carries the launch-wide fields.
template <typename T, typename VEL>
int batch_launch(wmibm_handle *h0, const Member<T> *dev_members, int nmembers, const KParams<T> &tmpl,
                 const StencilConfig &c, int max_nx, int wall_blocks, int form, cudaStream_t stream)
{
    KParams<T> p = tmpl;
    p.list = dev_members;
    p.nmembers = nmembers;
    p.stages = c.stages;
    p.ncons = c.consumer_warps;
    if (form == 5) return launch_stencil_ty<T, VEL, 0, kInterleaved>(h0, p, c, stream, false, max_nx);
    if (form == 6) return launch_stencil_ty<T, VEL, 0, kWarpSpec>(h0, p, c, stream, false, max_nx);
    // two chunks of 2 x 256 records in shared memory, then the member table
    // (3 offsets and 3 pointers a member, 8 bytes each, and two end entries)
    const size_t chunks = 2 * 2 * 256 * sizeof(typename RecOf<T>::type);
    const size_t wsmem = chunks + (size_t)(6 * nmembers + 2) * 8;
    const size_t wsmem_max = chunks + (size_t)(6 * kMaxBatchMembers + 2) * 8;
    static int per_sm = 0;                 // once per instantiation and process (at the largest table)
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_wall_batch<T, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)wsmem_max);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wall_batch<T, VEL>, 256, wsmem_max);
        if (e != cudaSuccess) return cuda_status(h0, e, "batch wall occupancy");
        if (per_sm < 1) per_sm = 1;
    }
    if (wall_blocks <= 0) {
        // one wave of resident blocks, or the tuning's blocks per SM
        const int bps = (c.wall_grid > 0 && c.wall_grid < per_sm) ? c.wall_grid : per_sm;
        wall_blocks = bps * h0->sm_count;
    }
    k_wall_batch<T, VEL><<<(unsigned)wall_blocks, 256, wsmem, stream>>>(p);
    int st = cuda_status(h0, cudaGetLastError(), "k_wall_batch launch");
    if (st) return st;
    return launch_stencil_ty<T, VEL, 0, kAfterWall>(h0, p, c, stream, true, max_nx);
}

template int batch_launch<float, float>(wmibm_handle *, const Member<float> *, int, const KParams<float> &,
                                        const StencilConfig &, int, int, int, cudaStream_t);
template int batch_launch<float, __nv_bfloat16>(wmibm_handle *, const Member<float> *, int, const KParams<float> &,
                                                const StencilConfig &, int, int, int, cudaStream_t);
template int batch_launch<double, double>(wmibm_handle *, const Member<double> *, int, const KParams<double> &,
                                          const StencilConfig &, int, int, int, cudaStream_t);

}  // namespace wmibm
