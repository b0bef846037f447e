// Batched ensembles: many terrains ("members") of uneven grid sizes stepped
// by the same two persistent launches (the wall kernel over the concatenated
// band records, then the pipelined force + mask kernel over the concatenated
// (member, strip, level) units).  The member descriptors live in device
// memory, so a step is graph-capturable and replays with the same fields.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "members.cuh"

using namespace wmibm;

struct wmibm_batch {
    int device;
    int count;
    int32_t dtype, vel_dtype;
    std::vector<wmibm_handle *> members;
    void *dev_members;          // Member<T>[count]
    double *bstats;             // [count][2][4]
    unsigned *ticket;
    int *status;
    int max_nx;
    std::vector<int> rows;      // rows per strip of each member's stencil
    uint32_t half_a, half_b;    // elements of the largest member's half-A and half-B stage slots
    int fields_set;
    wmibm_tuning tuning;
    StencilConfig cfg;
    int64_t clean_total, dirty_total, rec_total, run_total, body_total;
    int64_t traffic[2];
    uint64_t wait_ns;
    int hold_release;
    std::vector<unsigned char> member0;   // host copy of member 0's descriptor (a batch of one
                                          // is launched with it as the single-terrain member)
    char err[512];
};

namespace {

int berr(wmibm_batch *b, int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
    return status;
}

int bcuda(wmibm_batch *b, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return WMIBM_OK;
    return berr(b, e == cudaErrorMemoryAllocation ? WMIBM_ENOMEM : WMIBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Tile shape of the batch: the widest members take `rows` x-rows per strip
// (tuning.rows, default 4); narrower members take proportionally more rows (at
// most 16, dividing ny) so that every member's stage carries about the same
// bytes.  The stage slots hold the largest member's stage halves; two unless the
// tuning sets them (the autotuner's pick on the measured ensembles: three blocks
// per SM).
bool batch_config(wmibm_batch *b, StencilConfig *out, std::vector<int> *rows_out, uint32_t *half_a,
                  uint32_t *half_b)
{
    const size_t es = elem_size(b->dtype);
    const int V = 16 / (int)es;
    const int base = b->tuning.rows > 0 ? b->tuning.rows : 4;
    if (!(base == 1 || base == 2 || base == 4)) return false;
    std::vector<int> rows;
    size_t ha = 0, hb = 0;
    for (auto *h : b->members) {
        if (h->nx % V != 0 || h->nz < 3 || h->ny < 3) return false;
        int target = (int)std::min<int64_t>(16, std::max<int64_t>(1, (int64_t)base * b->max_nx / h->nx));
        int ty = 0;
        for (int t = target; t >= 1; --t)
            if (h->ny % t == 0 && h->ny >= t + 2) {
                ty = t;
                break;
            }
        if (ty == 0) return false;
        rows.push_back(ty);
        ha = std::max(ha, (size_t)(3 * ty + 4) * h->nx);
        hb = std::max(hb, (size_t)(3 * ty + 2) * h->nx);
    }
    auto ring_bytes = [&](int s) { return ((size_t)s * ha + (size_t)(s + 1) * hb) * es; };
    int stages = b->tuning.stages;
    if (stages == 0) stages = 2;
    if (stages < 2 || stages > 8 || ring_bytes(stages) + 256 > 200 * 1024) return false;
    out->rows = 0;                 // per member
    out->stages = stages;
    out->consumer_warps = b->tuning.consumer_warps > 0 ? b->tuning.consumer_warps : 4;
    out->wall_warps = b->tuning.wall_warps;
    out->blocks_per_sm = b->tuning.blocks_per_sm;
    out->wall_chunk = b->tuning.wall_chunk;
    // a batch that was never tuned also takes its units in runs of at least 16 (the
    // autotuner's pick on the measured ensembles; a fixed share per block left a
    // spread of about 50 us between the first and the last block)
    const wmibm_tuning none = {};
    const bool untuned = memcmp(&b->tuning, &none, sizeof(none)) == 0;
    out->dyn_chunk = untuned ? 16 : b->tuning.dyn_chunk;
    out->wall_grid = b->tuning.wall_grid;
    if (b->tuning.wall_grid < 0 || b->tuning.wall_grid > 32) return false;
    // one launch (force_path 0 or 6: wall warps; 5: interleaved wall stages) or two launches (3)
    if (b->tuning.dyn_chunk < 0 || b->tuning.dyn_chunk > 4096) return false;
    const int fp = b->tuning.force_path;
    if (!(fp == 0 || fp == 3 || fp == 5 || fp == 6)) return false;
    if (fp != 3 && fp != 5 && 1 + out->consumer_warps + (out->wall_warps > 0 ? out->wall_warps : 3) > 16)
        return false;
    if (1 + out->consumer_warps > 16) return false;
    *rows_out = rows;
    *half_a = (uint32_t)ha;
    *half_b = (uint32_t)hb;
    return true;
}

template <typename T>
int upload_members(wmibm_batch *b, const wmibm_member_fields *fields, cudaStream_t stream)
{
    std::vector<Member<T>> host(b->count);
    int64_t c_off = 0, d_off = 0, r_off = 0, run_off = 0, body_off = 0;
    for (int m = 0; m < b->count; ++m) {
        wmibm_handle *h = b->members[m];
        const wmibm_member_fields &fl = fields[m];
        fill_member<T>(h, host[m], (const void *const *)fl.tau, fl.f, fl.u, fl.v, fl.w, h->logz0, nullptr, 0.0,
                       b->rows[m]);
        Member<T> &mm = host[m];
        mm.c_off = c_off;
        mm.d_off = d_off;
        mm.r_off = r_off;
        mm.run_off = run_off;
        mm.body_off = body_off;
        c_off += (int64_t)mm.nstrips * (mm.da + (mm.nz - mm.db));
        d_off += (int64_t)mm.nstrips * (mm.db - mm.da);
        r_off += mm.nb_w + mm.nb_uv;
        run_off += mm.nr_w + mm.nr_uv;
        body_off += mm.nbody_w + mm.nbody_uv;
    }
    b->clean_total = c_off;
    b->dirty_total = d_off;
    b->rec_total = r_off;
    b->run_total = run_off;
    b->body_total = body_off;
    b->member0.resize(sizeof(Member<T>));
    memcpy(b->member0.data(), &host[0], sizeof(Member<T>));
    cudaError_t e = cudaMemcpyAsync(b->dev_members, host.data(), sizeof(Member<T>) * b->count,
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return bcuda(b, e, "upload member descriptors");
}

template <typename T, typename VEL>
int step_impl(wmibm_batch *b, wmibm_band_stats *stats, int do_mask, cudaStream_t stream)
{
    KParams<T> p = {};
    p.clean_total = b->clean_total;
    p.dirty_total = b->dirty_total;
    p.rec_total = b->rec_total;
    p.run_total = b->run_total;
    p.body_total = b->body_total;
    p.status = b->status;
    p.do_mask = do_mask;
    p.partials = nullptr;
    p.ticket = b->ticket;
    p.stats = stats;
    p.bstats = b->bstats;
    p.half_a = b->half_a;
    p.half_b = b->half_b;
    if (b->count == 1) memcpy(&p.one, b->member0.data(), sizeof(Member<T>));   // kernels read p.one then
    p.wall_done = b->ticket + 1;
    p.exit_ticket = b->ticket + 2;
    p.wait_ns = b->wait_ns;
    p.hold_release = b->hold_release;
    const int wall_blocks = 0;   // one wave of resident blocks
    // untuned: two launches, the form the autotuner keeps on the measured ensembles
    const int form = b->tuning.force_path == 0 ? 3 : b->tuning.force_path;
    int st = batch_launch<T, VEL>(b->members[0], (const Member<T> *)b->dev_members, b->count, p, b->cfg, b->max_nx,
                                  wall_blocks, form, stream);
    if (st) return berr(b, st, "%s", b->members[0]->err);
    return WMIBM_OK;
}

}  // namespace

extern "C" int wmibm_batch_create(wmibm_batch **out, wmibm_handle *const *members, int32_t count, void *stream)
{
    ApiRange nvtx_range("wmibm_batch_create");
    if (!out) return WMIBM_EINVAL;
    *out = nullptr;
    if (!members || count < 1 || count > kMaxBatchMembers) return WMIBM_EINVAL;
    for (int m = 0; m < count; ++m)
        if (!members[m]) return WMIBM_EINVAL;
    const wmibm_handle *h0 = members[0];
    for (int m = 1; m < count; ++m)
        if (members[m]->device != h0->device || members[m]->dtype != h0->dtype ||
            members[m]->vel_dtype != h0->vel_dtype)
            return WMIBM_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h0->device) return WMIBM_ESTATE;
    fault_arm();

    wmibm_batch *b = fault_fires() ? nullptr : new (std::nothrow) wmibm_batch();
    if (!b) return WMIBM_ENOMEM;
    b->device = h0->device;
    fault_wait_settings(&b->wait_ns, &b->hold_release);
    b->count = count;
    b->dtype = h0->dtype;
    b->vel_dtype = h0->vel_dtype;
    b->members.assign(members, members + count);
    b->max_nx = 0;
    for (auto *h : b->members) b->max_nx = std::max(b->max_nx, (int)h->nx);
    const size_t msize = b->dtype == WMIBM_F64 ? sizeof(Member<double>) : sizeof(Member<float>);
    cudaError_t e = dev_alloc(&b->dev_members, msize * count);
    if (e == cudaSuccess) e = dev_alloc(&b->bstats, sizeof(double) * 8 * count);
    // [0] last-block ticket of the batch wall kernel; [1] wall-done and [2] exit
    // counters of the single launch; [4..7] the two 64-bit counters of the dynamic
    // dispensing (all back at 0 after every launch)
    if (e == cudaSuccess) e = dev_alloc(&b->ticket, 8 * sizeof(unsigned));
    if (e == cudaSuccess) e = dev_alloc(&b->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bstats, 0, sizeof(double) * 8 * count, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ticket, 0, 8 * sizeof(unsigned), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess || !batch_config(b, &b->cfg, &b->rows, &b->half_a, &b->half_b)) {
        cudaFree(b->dev_members);
        cudaFree(b->bstats);
        cudaFree(b->ticket);
        cudaFree(b->status);
        delete b;
        if (e == cudaErrorMemoryAllocation) return WMIBM_ENOMEM;
        return e != cudaSuccess ? WMIBM_ECUDA : WMIBM_EINVAL;
    }
    int64_t wall_bytes = 0, force_bytes = 0;
    for (auto *h : b->members) {
        wall_bytes += h->traffic[0];
        force_bytes += h->traffic[1] + h->traffic[2];
    }
    b->traffic[0] = wall_bytes;
    b->traffic[1] = force_bytes;
    *out = b;
    return WMIBM_OK;
}

extern "C" int wmibm_batch_set_fields(wmibm_batch *b, const wmibm_member_fields *fields, void *stream)
{
    ApiRange nvtx_range("wmibm_batch_set_fields");
    if (!b) return WMIBM_EINVAL;
    if (!fields) return berr(b, WMIBM_EINVAL, "NULL fields");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return berr(b, WMIBM_ESTATE, "current device is not the batch's device");
    for (int m = 0; m < b->count; ++m) {
        const wmibm_member_fields &fl = fields[m];
        if (!fl.u || !fl.v || !fl.w) return berr(b, WMIBM_EINVAL, "member %d: NULL velocity", m);
        for (int a = 0; a < 6; ++a)
            if (!fl.tau[a] || !aligned16(fl.tau[a]))
                return berr(b, WMIBM_EINVAL, "member %d: stress %d NULL or not 16-byte aligned", m, a);
        for (int a = 0; a < 3; ++a)
            if (!fl.f[a] || !aligned16(fl.f[a]))
                return berr(b, WMIBM_EINVAL, "member %d: force %d NULL or not 16-byte aligned", m, a);
    }
    int st = b->dtype == WMIBM_F64 ? upload_members<double>(b, fields, (cudaStream_t)stream)
                                   : upload_members<float>(b, fields, (cudaStream_t)stream);
    if (st == WMIBM_OK) b->fields_set = 1;
    return st;
}

extern "C" int wmibm_batch_set_tuning(wmibm_batch *b, const wmibm_tuning *t)
{
    ApiRange nvtx_range("wmibm_batch_set_tuning");
    if (!b || !t) return WMIBM_EINVAL;
    wmibm_tuning old = b->tuning;
    b->tuning = *t;
    StencilConfig c;
    std::vector<int> rows;
    uint32_t ha = 0, hb = 0;
    if (!batch_config(b, &c, &rows, &ha, &hb)) {
        b->tuning = old;
        return berr(b, WMIBM_EINVAL, "tuning does not fit every member");
    }
    b->cfg = c;
    b->rows = rows;
    b->half_a = ha;
    b->half_b = hb;
    b->fields_set = 0;       // unit offsets depend on the rows per strip: set the fields again
    return WMIBM_OK;
}

static int batch_run(wmibm_batch *b, wmibm_band_stats *stats, int do_mask, void *stream)
{
    if (!b) return WMIBM_EINVAL;
    if (!b->fields_set) return berr(b, WMIBM_ESTATE, "wmibm_batch_set_fields must be called first");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return berr(b, WMIBM_ESTATE, "current device is not the batch's device");
    if (b->dtype == WMIBM_F64) return step_impl<double, double>(b, stats, do_mask, (cudaStream_t)stream);
    if (b->vel_dtype == WMIBM_BF16)
        return step_impl<float, __nv_bfloat16>(b, stats, do_mask, (cudaStream_t)stream);
    return step_impl<float, float>(b, stats, do_mask, (cudaStream_t)stream);
}

extern "C" int wmibm_batch_step(wmibm_batch *b, wmibm_band_stats *stats, void *stream)
{
    ApiRange nvtx_range("wmibm_batch_step");
    return batch_run(b, stats, 1, stream);
}

extern "C" int wmibm_batch_wall_stress_force(wmibm_batch *b, wmibm_band_stats *stats, void *stream)
{
    ApiRange nvtx_range("wmibm_batch_wall_stress_force");
    return batch_run(b, stats, 0, stream);
}

extern "C" int wmibm_batch_device_status(wmibm_batch *b, int32_t *out, void *stream)
{
    ApiRange nvtx_range("wmibm_batch_device_status");
    if (!b) return WMIBM_EINVAL;
    if (!out) return berr(b, WMIBM_EINVAL, "NULL output");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return berr(b, WMIBM_ESTATE, "current device is not the batch's device");
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch device status");
    *out = v == 0 ? WMIBM_OK : WMIBM_ETIMEOUT;
    return WMIBM_OK;
}

extern "C" int64_t wmibm_batch_traffic_bytes(const wmibm_batch *b, int32_t which)
{
    if (!b || which < 0 || which > 1) return -1;
    return b->traffic[which];
}

extern "C" int64_t wmibm_batch_points(const wmibm_batch *b)
{
    if (!b) return -1;
    int64_t n = 0;
    for (auto *h : b->members) n += h->n;
    return n;
}

extern "C" const char *wmibm_batch_last_error(const wmibm_batch *b) { return b ? b->err : ""; }

extern "C" void wmibm_batch_destroy(wmibm_batch *b)
{
    ApiRange nvtx_range("wmibm_batch_destroy");
    if (!b) return;
    cudaDeviceSynchronize();
    cudaFree(b->dev_members);
    cudaFree(b->bstats);
    cudaFree(b->ticket);
    cudaFree(b->status);
    delete b;
}
