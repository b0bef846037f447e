// Launch descriptors shared by the stencil / wall kernels (stencil.cu) and the
// batch API (batch.cu): one Member per terrain of a launch.
#pragma once

#include "internal.cuh"

namespace wmibm {

// One terrain of a launch: its fields and its precomputed lists.
template <typename T>
struct Member {
    const T *tau[6];              // txx txy tyy tzz txz tyz (the wall kernel writes band / solid entries)
    T *f[3];
    void *u, *v, *w;
    int32_t nx, ny, nz, nstrips, rows;   // rows: x-rows per strip of the stencil
    T cx, cy, cz;                 // 1/(2 dx), 1/(2 dy), 1/dz
    int32_t da, db;               // dirty levels [da, db)
    int64_t c_off, d_off;         // first index in the launch's clean / dirty unit spaces
    const void *rec;              // band records (w-band first)
    int64_t nb_w, nb_uv, r_off;   // band counts; first index in the record space
    int64_t nzc_w, nzc_uv;        // band nodes whose sample point's level is clamped (reported in the stats)
    const int2 *runs_w, *runs_uv; // solid runs along x
    int64_t nr_w, nr_uv, run_off;
    const int32_t *body_w, *body_uv;
    int64_t nbody_w, nbody_uv, body_off;
    const T *gpx, *gpy, *gpz;     // body mask: 3 dt/2 grad p, or NULL
    T mask_c;
    const T *logz0;               // optional per-cell log z0
    T log_phi_c, kappa2;
};

template <typename T>
struct KParams {
    Member<T> one;                // the member of a single-terrain launch (nmembers == 1)
    const Member<T> *list;        // device array of members (nmembers > 1)
    int nmembers;
    int64_t clean_total, dirty_total, rec_total, run_total, body_total;
    int stages, ncons;            // stages: depth of the ring of half A (half B has one more slot)
    uint32_t half_a, half_b;      // elements of a half-A and a half-B slot (the largest member's)
    int *status;
    int do_mask;
    // statistics: single terrain -> per-block partials reduced by the last block;
    // batch -> per-member accumulators (scratch) converted by the last block
    T *partials;
    unsigned *ticket;
    wmibm_band_stats *stats;
    double *bstats;               // batch: [nmembers][2][4] (sum, sum^2, -min bits, max bits)
    // fused single-terrain step (wall phase inside the stencil launch): blocks that
    // finished their wall share, and blocks that finished the launch (both back at 0
    // after every launch)
    unsigned *wall_done;
    unsigned *exit_ticket;
    // single terrain, statistics by reduction: the FP64 accumulator (handle-owned,
    // kept at 0 between calls) and whether this launch converts it into stats
    double *sacc;
    int emit_stats;
    // single-launch stage: 0 = every block's consumers evaluate a share of the wall
    // model first; > 0 = blocks [0, wall_blocks) only evaluate the wall model and
    // the others only stream the stencil; -1 = dedicated, chosen at launch
    int wall_blocks;
    // interleaved single-launch stage (interleave != 0): the band records, cut
    // into wall_items slices of wall_chunk records, are stages of the stencil
    // pipeline of every block (see StageIter)
    int interleave;
    int wall_chunk;
    int64_t wall_items;
    // warp-specialized single-launch stage: warps [1 + ncons, 1 + ncons + wall_warps)
    // of every block evaluate the block's slice of the band records and solid runs
    int wall_warps;
    // dynamic dispensing (dyn_chunk > 0): the producers take runs of dyn_chunk units
    // from the counters dyn_ctr[0] (clean units) and dyn_ctr[1] (dirty units), back
    // at 0 after every launch, instead of a fixed share per block
    int dyn_chunk;
    unsigned long long *dyn_ctr;
    // bounded waits give up after wait_ns; hold_release (a test of the failure path,
    // read from the environment at init) keeps the single-launch forms from counting
    // their blocks into wall_done, so that the waits on it run out
    uint64_t wait_ns;
    int hold_release;
};

template <typename T>
void fill_member(const wmibm_handle *h, Member<T> &m, const void *const tau[6], void *const f[3], void *u, void *v,
                 void *w, const void *logz0, const void *const gradp[3], double dt, int rows);

template <typename T, typename VEL>
int batch_launch(wmibm_handle *h0, const Member<T> *dev_members, int nmembers, const KParams<T> &tmpl,
                 const StencilConfig &c, int max_nx, int wall_blocks, int form, cudaStream_t stream);

bool stencil_config(const wmibm_handle *h, const void *const tau[6], void *const f[3], StencilConfig *out);

constexpr int kMaxBatchMembers = 256;

}  // namespace wmibm
