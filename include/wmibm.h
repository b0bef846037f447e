/*
 * wmibm.h - C ABI of libwmibm.so, the sm_103a CUDA implementation of the
 * per-time-step stress stage of the simplified wall-modeled immersed boundary
 * method (Liu & Stevens, arXiv:2006.03343, Sec. 3).
 *
 * Grid (Sec. 2.4, Eq. 12): nx x ny x nz nodes, dx = lx/nx, dy = ly/ny,
 * dz = lz/(nz-1).  Every field is a dense array [k][j][i] (i fastest),
 * nx*ny*nz elements, contiguous, on the device of the handle.
 *   uv-node (i,j,k) at (i dx, j dy, (k+1/2) dz): u, v, txx, txy, tyy, tzz, fx, fy
 *   w-node  (i,j,k) at (i dx, j dy, k dz):       w, txz, tyz, fz
 * The uv level k = nz-1 lies above the lid (ghost level).
 *
 * Stress arrays are passed as an array of 6 pointers in the order
 *   tau[0..5] = txx, txy, tyy, tzz, txz, tyz.
 *
 * Conventions for every call:
 *   - the caller owns every field buffer; the handle owns its index lists and
 *     band records (copied/derived at init) and frees them in wmibm_destroy;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     work is enqueued on it and the call returns without waiting, except
 *     wmibm_init, which synchronises `stream` once to read back list sizes;
 *   - the calling thread's current CUDA device must be the handle's device;
 *   - the return value is a status code below; on failure nothing further is
 *     enqueued and wmibm_last_error(h) describes the problem;
 *   - calls on one handle must not overlap on the GPU (they share the handle's
 *     reduction scratch): use one stream per handle, or order the streams.
 */
#ifndef WMIBM_H
#define WMIBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define WMIBM_OK 0
#define WMIBM_EINVAL 1    /* invalid argument (sizes, NaN in phi, z0 >= phi_c, ...) */
#define WMIBM_ENOMEM 2    /* device or host allocation failed */
#define WMIBM_ECUDA 3     /* a CUDA runtime call or kernel launch failed */
#define WMIBM_ESTATE 4    /* wrong device, or a call the handle's mode does not allow */
#define WMIBM_ETIMEOUT 5  /* a bounded device-side wait gave up */

/* element types */
#define WMIBM_F32 0
#define WMIBM_F64 1
#define WMIBM_BF16 2

/* list selectors for wmibm_list_size / wmibm_export_list */
#define WMIBM_LIST_BAND_W 0      /* w-nodes with -phi_b <= phi <= phi_b      (Sec. 3.3) */
#define WMIBM_LIST_BAND_UV 1     /* uv-nodes with 0 <= phi <= 2 phi_b        (Sec. 3.3) */
#define WMIBM_LIST_SOLID_W 2     /* w-nodes with phi < -phi_b: txz = tyz = 0 (Sec. 3.3) */
#define WMIBM_LIST_SOLID_UV 3    /* uv-nodes with phi < 0: txx..tzz = 0      (Sec. 3.3) */
#define WMIBM_LIST_BODY_W 4      /* w-nodes with phi <= 0: masked w          (Sec. 3.2, Eq. 27) */
#define WMIBM_LIST_BODY_UV 5     /* uv-nodes with phi <= 0: masked u, v      (Sec. 3.2, Eq. 27) */

typedef struct wmibm_grid {
    int32_t nx, ny, nz;     /* nodes per direction; nz >= 3 */
    double lx, ly, lz;      /* domain lengths, > 0 */
} wmibm_grid;

typedef struct wmibm_opts {
    double phi_b;           /* half band width; <= 0 selects dz/2 (2 phi_b = dz, Sec. 3.3) */
    double kappa;           /* von Karman constant; <= 0 selects 0.4 (Sec. 2.2) */
    int32_t dtype;          /* WMIBM_F32 or WMIBM_F64: type of tau, f, grad p and of the arithmetic */
    int32_t vel_dtype;      /* storage type of u, v, w: equal to dtype, or WMIBM_BF16 when dtype is F32 */
    int32_t zclamp;         /* sample points x_c above the top or below the bottom physical level of a
                               grid (Sec. 3.3 interpolation): WMIBM_ZCLAMP_CLAMP (0) clamps their level
                               (reading R3) and counts them in wmibm_band_stats.n_zclamped;
                               WMIBM_ZCLAMP_REJECT (1) makes wmibm_init fail with EINVAL instead */
    int32_t own_x0, own_x1; /* 0, 0: the handle owns every node.  Otherwise 0 <= own_x0 < own_x1 <= nx:
                               it owns the nodes with own_x0 <= i < own_x1, and the others are halo
                               planes of a slab of a larger domain cut along x: they serve the normals
                               and stencils of owned nodes but are never band, solid or body nodes, so
                               every per-node output there is left to the slab that owns them */
} wmibm_opts;

#define WMIBM_ZCLAMP_CLAMP 0
#define WMIBM_ZCLAMP_REJECT 1

/* Band statistics of one wall-stress pass, one record per band (w, then uv). */
typedef struct wmibm_band_stats {
    int64_t count;          /* band nodes */
    double sum_tw;          /* sum of tau_w = -[kappa U_r / ln(phi_c/z0)]^2  (Eq. 28) */
    double sum_tw2;         /* sum of tau_w^2 */
    double min_tw;          /* most negative tau_w (0 for an empty band) */
    double max_ur;          /* largest tangential speed |U_r| (0 for an empty band) */
    int64_t n_zclamped;     /* band nodes whose sample point x_c had its level clamped to the physical
                               levels of the uv-grid or the w-grid (fixed by phi: counted at init) */
} wmibm_band_stats;

typedef struct wmibm_handle wmibm_handle;

/*
 * wmibm_init - one-time set-up for one terrain (Sec. 3.1 and Sec. 3.3: the
 * distance phi, the normals and the node classes are fixed per geometry, so
 * they are computed here once).
 *   out      : receives the new handle
 *   g        : grid; nx*ny*nz must be < 2^31
 *   phi_uv   : HOST, nx*ny*nz doubles: signed distance at the uv-nodes (+ fluid, - solid)
 *   phi_w    : HOST, nx*ny*nz doubles: signed distance at the w-nodes
 *   z0       : HOST: one double (z0_is_field = 0) or nx*ny*nz doubles, the roughness
 *              of cell (i,j,k), shared by uv-node and w-node (i,j,k); 0 < z0 < phi_c
 *   phi_c    : distance above the surface at which the velocity is sampled
 *              (Sec. 3.3, phi_c >= 2 phi_b)
 *   opts     : NULL for defaults (F32, phi_b = dz/2, kappa = 0.4, zclamp = CLAMP)
 * The inputs are copied; the handle keeps no pointer to them.  On the GPU (in
 * FP64) it classifies every node, computes n = grad(phi)/|grad(phi)| by central
 * differences, builds ascending index lists of the band, solid and body nodes
 * and, per band node, the interpolation stencil of x_c = x + (phi_c - phi) n
 * and the factor kappa^2 / ln^2(phi_c/z0).
 * Errors: EINVAL (bad sizes, non-finite phi, z0 out of range, phi_c < 2 phi_b,
 * a clamped sample point with zclamp = REJECT), ENOMEM, ECUDA.  On error *out is NULL.
 */
int wmibm_init(wmibm_handle **out, const wmibm_grid *g, const double *phi_uv, const double *phi_w,
               const double *z0, int32_t z0_is_field, double phi_c, const wmibm_opts *opts, void *stream);

/*
 * wmibm_wall_stress - the wall model at every band node (Sec. 3.3, Eq. 28 and
 * the rotation tau_ij = a_im a_jn tau'_mn).
 *   u, v, w  : DEVICE velocity fields (vel_dtype), read only
 *   tau      : DEVICE stresses (dtype), in/out: fluid entries are left untouched,
 *              band entries are overwritten (txz, tyz on w-band nodes; txx, txy,
 *              tyy, tzz on uv-band nodes), solid entries are set to 0
 *   stats    : NULL, or DEVICE-accessible wmibm_band_stats[2] (w-band, uv-band),
 *              written on the stream after the wall kernel; sums are accumulated
 *              per block in the path dtype, then across blocks in FP64 with
 *              atomic reductions (so FP64 sums may differ in the last bits from
 *              call to call; counts, minima and maxima are exact)
 * Errors: EINVAL (NULL field pointer), ESTATE, ECUDA.
 */
int wmibm_wall_stress(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                      wmibm_band_stats *stats, void *stream);

/*
 * wmibm_force - the forcing f = -div(tau) on the staggered grid (Eq. 2 and
 * Eq. 18, vertical differences of Eqs. 15-16; horizontal derivatives are
 * second-order central differences, periodic).
 *   tau      : DEVICE, 6 stress fields (dtype), read only
 *   fx, fy   : DEVICE uv-node fields (dtype), written everywhere; 0 on the ghost level
 *   fz       : DEVICE w-node field (dtype), written everywhere; 0 on the floor and lid
 * Errors: EINVAL, ESTATE, ECUDA.
 */
int wmibm_force(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, void *stream);

/*
 * wmibm_force_spectral - the forcing f = -div(tau) with the paper's own
 * horizontal scheme: x and y derivatives pseudo-spectral (Sec. 2.4, Eqs. 13-14:
 * the derivative of each periodic plane is the sum over (k_x, k_y) of i k A-hat
 * e^{i(k_x x + k_y y)}), vertical differences as in wmibm_force (Eqs. 15-16).
 * The Nyquist wavenumber of each direction carries no first derivative.
 * Arguments, layout and boundary rows as in wmibm_force.  One persistent launch
 * (FFT lines in shared memory, FP32 or FP64 as the handle's dtype); tau and
 * f must not overlap.
 * Requires nx and ny powers of two in [2, 2048] for FP32, [2, 1024] for FP64:
 * otherwise EINVAL, before any GPU work.  Errors: EINVAL, ESTATE, ECUDA.
 */
int wmibm_force_spectral(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, void *stream);

/*
 * wmibm_sgs_wall_terms - the per-node wall term of Mason's damping (Sec. 2.2,
 * Eq. 7 with n = 2) for wmibm_sgs_stress and wmibm_sgs_force: 1/[kappa (phi + z0)]^2
 * at fluid nodes (uv-grid phi > 2 phi_b, w-grid phi > phi_b: neither band nor
 * solid, Sec. 3.3), -1 at band nodes, -2 at solid nodes.  Computed on the host
 * in FP64, stored in the handle's dtype.
 *   phi_uv, phi_w : HOST, N each, FP64, the same fields as given to wmibm_init
 *   z0            : HOST, scalar (z0_is_field = 0) or per-cell [k][j][i] (1)
 *   wt_uv, wt_w   : DEVICE, N each (dtype), caller-owned, written
 * Synchronizes the stream; call it once per geometry, before any stream capture.
 * Errors: EINVAL, ENOMEM, ESTATE, ECUDA.
 */
int wmibm_sgs_wall_terms(wmibm_handle *h, const double *phi_uv, const double *phi_w, const double *z0,
                         int32_t z0_is_field, void *wt_uv, void *wt_w, void *stream);

/*
 * wmibm_sgs_stress - the Smagorinsky sub-grid stress with Mason's wall damping
 * (Sec. 2.2, Eqs. 4-7) written into tau at fluid nodes: tau_ij = -2 nu_t S_ij,
 * nu_t = lambda^2 |S|, |S| = sqrt(2 S:S), 1/lambda^2 = 1/(C_s l)^2 + wall term,
 * l = (dx dy dz)^(1/3), z of Eq. 7 = the node's phi.  S11, S22, S12 (periodic
 * central differences) and S33 (Eq. 16) on uv-nodes, S13, S23 on w-nodes (Eq. 15);
 * |S| on a uv-node averages S13, S23 of the w-levels around it (the floor repeats
 * the level above, the lid counts 0), on a w-node S11, S22, S33, S12 of the
 * uv-levels around it.  Band and solid entries, the ghost uv-level and the floor
 * w-level are left as they are (run wmibm_wall_stress afterwards for the band);
 * the lid's fluid tau_xz, tau_yz become 0 (Eq. 10).
 *   u, v, w       : DEVICE velocity (vel_dtype), read only
 *   wt_uv, wt_w   : DEVICE wall terms from wmibm_sgs_wall_terms
 *   tau           : 6 DEVICE stress fields (dtype), written at fluid nodes
 *   cs            : the Smagorinsky coefficient C_s (the paper uses 0.16), > 0
 * Neither this call nor wmibm_wall_stress reads tau, and the entries they write
 * are disjoint (fluid here; band and solid there), so the two may run at the
 * same time on two streams of the handle's device, with wmibm_force after both.
 * Errors: EINVAL, ESTATE, ECUDA.
 */
int wmibm_sgs_stress(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv,
                     const void *wt_w, void *const tau[6], double cs, void *stream);

/*
 * wmibm_sgs_force - the forcing f = -div(tau) of wmibm_force with the fluid stress
 * formed on the fly from the velocity, as wmibm_sgs_stress would write it, in one
 * pass that never writes tau: at each node tau is the Smagorinsky stress (fluid),
 * the value in tau (band: call wmibm_wall_stress first; and the floor w-level),
 * or 0 (solid; the lid's fluid tau_xz, tau_yz).  Equal to wmibm_sgs_stress, then
 * wmibm_wall_stress, then wmibm_force, up to rounding, with about 32 instead of
 * about 80 bytes per node moved.
 *   u, v, w, wt_uv, wt_w, cs : as in wmibm_sgs_stress
 *   tau           : 6 DEVICE stress fields (dtype), read at band nodes and on the floor only
 *   fx, fy, fz    : DEVICE forcing (dtype), written everywhere (0 on the ghost level, floor and lid as in
 *                   wmibm_force); must not overlap tau, the velocity or the wall terms
 * Errors: EINVAL, ESTATE, ECUDA.
 */
int wmibm_sgs_force(wmibm_handle *h, const void *u, const void *v, const void *w, const void *wt_uv,
                    const void *wt_w, const void *const tau[6], void *fx, void *fy, void *fz, double cs, void *stream);

/*
 * wmibm_heightfield_sdf - the signed distance phi of Sec. 3.1 (+d in the fluid,
 * -d in the solid, d the minimum distance to the immersed boundary) for terrain
 * given as heights, on both grids, ready for wmibm_init.  The boundary is the
 * piecewise-linear surface through the heights: cell [i, i+1] x [j, j+1] is
 * split along its (i, j)-(i+1, j+1) diagonal into two flat triangles, periodic
 * in x and y.  The sign is that of z - h[j][i] (the node's column passes
 * through a vertex).  Nodes within `reach` of the surface get the exact
 * distance; all others keep z - h[j][i], whose magnitude exceeds the reach, so
 * class thresholds below the reach (0, phi_b, 2 phi_b, phi_c) see exact values.
 * No handle: it runs before wmibm_init, which takes phi on the host.
 *   g              : grid (nx, ny >= 1, nz >= 3, nx*ny*nz < 2^31, lengths > 0)
 *   height         : DEVICE, ny*nx finite doubles, h[j][i] at (i dx, j dy), read only
 *   reach          : > 0; the window it spans may hold at most 1024 cells
 *                    (4 ceil(reach/dx) ceil(reach/dy)) and 128 in each direction
 *   phi_uv, phi_w  : DEVICE, nx*ny*nz doubles each, [k][j][i], written everywhere;
 *                    uv-node (i, j, k) at z = (k + 1/2) dz, w-node at z = k dz
 *   stream         : CUDA stream (NULL = legacy default)
 * FP64 throughout; the work is queued on the stream (no synchronisation).
 * Errors (wmibm_last_error(NULL) has the text): EINVAL (NULL pointer, bad grid,
 * reach not finite or <= 0 or too wide, phi_uv == phi_w), ECUDA.
 */
int wmibm_heightfield_sdf(const wmibm_grid *g, const double *height, double reach, double *phi_uv, double *phi_w,
                          void *stream);

/*
 * wmibm_spectral_shape - the tile of wmibm_force_spectral's launch (host query):
 * out[0] rows per row unit, out[1] columns per column unit, out[2] z-levels per
 * chunk of the dispense order, out[3] shared-memory bytes per block.
 * Returns EINVAL for a NULL argument or a grid without spectral support.
 */
int wmibm_spectral_shape(const wmibm_handle *h, int64_t out[4]);

/*
 * wmibm_mask - the immersed-boundary velocity condition (Sec. 3.2, Eq. 27):
 * where phi <= 0 (each component on its own grid) the velocity becomes
 * 3 dt/2 * grad p, or 0 when gradp is NULL; elsewhere it is untouched.
 *   u, v, w  : DEVICE velocity fields (vel_dtype), in/out
 *   gradp    : NULL, or 3 DEVICE fields (dtype): dp/dx, dp/dy on uv-nodes, dp/dz on w-nodes
 * Errors: EINVAL, ESTATE, ECUDA.
 */
int wmibm_mask(wmibm_handle *h, void *u, void *v, void *w, const void *const gradp[3], double dt, void *stream);

/*
 * wmibm_step - wmibm_wall_stress, wmibm_force and wmibm_mask in that order on
 * one stream: one pass of the whole per-step stress stage, with the same results
 * as the three calls.  Where the pipelined stencil takes the grid (see
 * wmibm_force_mask) and tuning.force_path is not 3, it is ONE cooperative launch:
 * in every block the consumer warps first evaluate the block's share of the
 * band nodes and solid runs while the producer streams the stencil stages that
 * read no band or solid node; stages that do wait (bounded) until every block
 * has finished its wall share; the body mask follows the forcing.  Otherwise
 * it is two launches (the wall-model kernel, then the force + mask kernel as
 * its programmatic dependent).  A cooperative launch needs all its blocks
 * resident: it fails with ECUDA if another context holds the SMs it needs.
 */
int wmibm_step(wmibm_handle *h, void *u, void *v, void *w, void *const tau[6], void *fx, void *fy, void *fz,
               const void *const gradp[3], double dt, wmibm_band_stats *stats, void *stream);

/*
 * wmibm_wall_stress_force - wmibm_wall_stress followed by wmibm_force on one
 * stream (same arguments and results as the two calls); one cooperative launch
 * under the same conditions as wmibm_step (without the body mask).
 */
int wmibm_wall_stress_force(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                            void *fx, void *fy, void *fz, wmibm_band_stats *stats, void *stream);

/*
 * wmibm_force_mask - wmibm_force followed by wmibm_mask, in one launch where the
 * grid allows the pipelined stencil (nx a multiple of 4 for F32 or 2 for F64,
 * ny >= 3, 16-byte aligned stress and force buffers, full x-rows that fit the
 * shared-memory stages): the kernel forms f and then applies Eq. 27 to u, v, w.
 * Otherwise the force and mask kernels run back to back.  Arguments as in
 * wmibm_force and wmibm_mask.
 */
int wmibm_force_mask(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, void *u, void *v,
                     void *w, const void *const gradp[3], double dt, void *stream);

/*
 * Launch tuning of the stencil kernels (what the autotuner sets).  Zero fields
 * mean "choose automatically".
 */
typedef struct wmibm_tuning {
    int32_t force_path;       /* 0 auto, 1 bulk-copy pipeline only, 2 direct-load kernel only,
                                 3 bulk-copy pipeline with the wall model always in a kernel of its
                                 own (no single-launch step), 4 as 1 with the single-launch step's
                                 wall model in dedicated blocks (one per SM) instead of a share of
                                 every block, 5 single launch with the band records cut into "wall
                                 items" of wall_chunk records, each a stage of the pipeline of the
                                 block that owns it, spread over the first half of its clean units,
                                 6 single launch with wall_warps extra warps in every block that
                                 evaluate the block's share of the band records while the producer
                                 and consumers stream the clean units.  A batch takes 0 (two
                                 launches, as 3), 3, 5 or 6 */
    int32_t rows;             /* pipeline: rows per strip, 1, 2 or 4 */
    int32_t stages;           /* pipeline: shared-memory stages, 2..8 */
    int32_t consumer_warps;   /* pipeline: warps forming f, 1..12 */
    int32_t wall_warps;       /* fused step: warps per block of the wall-model kernel, 1..8 */
    int32_t blocks_per_sm;    /* pipeline: cap on resident blocks per SM */
    int32_t direct_bx;        /* direct-load kernel: vectors per block row */
    int32_t direct_by;        /* direct-load kernel: rows per block */
    int32_t direct_kc;        /* direct-load kernel: levels per thread */
    int32_t wall_chunk;       /* interleaved single launch (force_path 5): band records per wall
                                 stage, capped by a stage buffer (0: two per consumer thread) */
    int32_t dyn_chunk;        /* pipelined stencil outside force_path 1, 4, 5: 0 gives every block a
                                 fixed share of the (strip, level) units; n > 0 lets the blocks take
                                 runs of units from a counter as they go (clean units, then dirty),
                                 each run a share of what is left but at least n units */
    int32_t wall_grid;        /* wall kernel of the two-launch forms (force_path 3, batch included):
                                 blocks per SM of its grid (0: as many as fit); fewer leave room on
                                 every SM for the stencil launch that follows as its programmatic
                                 dependent, whose clean units then stream meanwhile */
} wmibm_tuning;

/* Sets / reads the tuning of handle h. EINVAL for out-of-range fields. */
int wmibm_set_tuning(wmibm_handle *h, const wmibm_tuning *t);
int wmibm_get_tuning(const wmibm_handle *h, wmibm_tuning *t);

/*
 * wmibm_device_status - reads and clears the handle's device status word, which
 * a kernel sets when one of its bounded waits gave up (ETIMEOUT).  Synchronises
 * `stream`.  *out receives WMIBM_OK or WMIBM_ETIMEOUT; the returned status is
 * that of the call itself.
 */
int wmibm_device_status(wmibm_handle *h, int32_t *out, void *stream);

/*
 * wmibm_wall_stress_noalloc - wmibm_wall_stress without any device allocation.
 * The paper has no counterpart: this is a deployment variant for callers that
 * cannot allocate device memory when they make the call -- code running while a
 * CUDA graph is being captured (cudaMalloc is not allowed there), plug-ins
 * whose host framework owns the device memory pool, real-time loops that must
 * not touch the allocator.  The handle itself must already exist (wmibm_init
 * allocates).
 *   Same arguments and results as wmibm_wall_stress (stats up to summation
 *   order).  The kernel's reduction scratch (per-block partial statistics and a
 *   ticket) is a static device array of 131,328 bytes that every GPU loading
 *   the library holds until the process exits.  The array bounds the kernel's
 *   blocks (2048); by choice, so that one call is one pass of that grid at two
 *   records a thread, at most 1,048,576 band nodes (w-band + uv-band) are
 *   accepted, and larger bands return EINVAL before any GPU work.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, and so does the first call
 *   after the device's context was made anew (cudaDeviceReset): make that first
 *   call before any stream capture.  All calls share the array and it keeps the
 *   last call's contents (the ticket is cleared on the stream before each
 *   launch): calls that overlap on the GPU, on any handle, race.  Host threads
 *   may make calls at the same time (the look-up is locked).
 */
int wmibm_wall_stress_noalloc(wmibm_handle *h, const void *u, const void *v, const void *w, void *const tau[6],
                              wmibm_band_stats *stats, void *stream);

/*
 * Adjoint (gradients of one stage).  The stage is the wall stress of Sec. 3.3
 * followed by f = -div(tau) (Eqs. 15-16, Eq. 18); the paper does not
 * differentiate it: this is the chain rule of that computation, for a scalar
 * L = sum over nodes of (gx fx + gy fy + gz fz) with the per-cell roughness
 * s = ln z0 as a parameter: C = kappa^2 / (ln phi_c - s)^2.
 *
 * wmibm_set_log_z0 - use a per-cell ln z0 field from now on.
 *   logz0 : DEVICE, nx*ny*nz elements of dtype, [k][j][i], the log roughness of
 *           cell (i,j,k), shared by its uv-node and w-node; every exp(s) must
 *           lie in (0, phi_c) (not checked).  The caller keeps the buffer alive
 *           and unchanged while the handle uses it.  NULL returns to the z0
 *           given at init.
 * Every later wmibm_wall_stress, wmibm_wall_stress_noalloc, wmibm_step,
 * wmibm_wall_stress_force and batch step of this handle computes C per node
 * from it.  The first call also builds the transpose of the band records'
 * trilinear gathers (host sort of 16 entries per band node, then upload; it
 * synchronizes `stream`), so make it before any stream capture.
 * Errors: EINVAL (misaligned logz0, more than 2^27 band nodes), ESTATE,
 * ENOMEM, ECUDA.
 */
int wmibm_set_log_z0(wmibm_handle *h, const void *logz0, void *stream);

/*
 * wmibm_backward - dL/du, dL/dv, dL/dw and dL/d(ln z0) of one stage.
 *   g      : DEVICE gx, gy (uv-grid) and gz (w-grid), dtype: the weights of L
 *   uvw    : DEVICE u, v, w (vel_dtype): the velocity the forward pass read
 *   du, dv, dw : DEVICE out, dtype, nx*ny*nz each: written everywhere (zero
 *            where no band stencil reaches)
 *   dlogz0 : DEVICE out (dtype, nx*ny*nz) or NULL: per cell, the sum of the
 *            contributions of its w-band and uv-band nodes (zero elsewhere);
 *            with no ln z0 field set, the derivative is taken at s = ln z0 of
 *            init
 * The fluid stresses pass through the stage and the solid ones are zero, so
 * neither depends on the velocity; the stress is not differentiated.  At a
 * band node with U_r = 0 the gradient is taken as zero.  Three kernels (the
 * per-node chain rule, then one gather per touched node in a fixed order) and
 * no atomics: the result is deterministic.  The first call builds the transpose
 * map if wmibm_set_log_z0 has not (synchronizing, as above).
 * Errors: EINVAL (NULL pointer), ESTATE, ENOMEM, ECUDA.
 */
int wmibm_backward(wmibm_handle *h, const void *const g[3], const void *const uvw[3], void *du, void *dv, void *dw,
                   void *dlogz0, void *stream);

/*
 * Batched ensembles: many terrains of uneven grid sizes stepped together.
 * The step of a batch is the per-step stage (wmibm_step without grad p) of
 * every member, done by two persistent launches over all members: the wall
 * kernel over the concatenated band records and solid runs, then the
 * pipelined force + body-mask kernel over the concatenated (member, strip,
 * level) units.  Member descriptors (field pointers) live in device memory, so
 * a step can be captured in a CUDA graph and replayed.
 */
typedef struct wmibm_batch wmibm_batch;

typedef struct wmibm_member_fields {
    void *u, *v, *w;        /* DEVICE velocity (vel_dtype), in/out (body mask) */
    void *tau[6];           /* DEVICE stresses (dtype), in/out, 16-byte aligned */
    void *f[3];             /* DEVICE forcing (dtype), out, 16-byte aligned */
} wmibm_member_fields;

/*
 * wmibm_batch_create - a batch over `count` (1..256) handles of one device with
 * the same dtype and vel_dtype.  The batch keeps the handle pointers (it does
 * not own them: destroy the batch first).  Every member must take the
 * pipelined stencil (nx a multiple of 4 for F32 or 2 for F64, ny >= 3) with a
 * common number of rows per strip.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA.
 */
int wmibm_batch_create(wmibm_batch **out, wmibm_handle *const *members, int32_t count, void *stream);

/* Sets the fields of every member (HOST array of count entries); synchronises
 * `stream` after uploading the descriptors.  Must precede wmibm_batch_step and
 * follow any wmibm_batch_set_tuning. */
int wmibm_batch_set_fields(wmibm_batch *b, const wmibm_member_fields *fields, void *stream);

/* Tile shape and form of the batch launches (force_path, rows, stages, consumer_warps,
 * wall_warps, blocks_per_sm, dyn_chunk, wall_grid used).  A batch that is never
 * tuned (every field 0) takes two launches, 4-row strips, two stages, four
 * consumer warps and runs of at least 16 units. */
int wmibm_batch_set_tuning(wmibm_batch *b, const wmibm_tuning *t);

/*
 * wmibm_batch_step - one step of every member (wall stress, force, mask).
 *   stats : NULL, or DEVICE wmibm_band_stats[count][2] (w-band, uv-band per member)
 * No host synchronisation; capturable in a CUDA graph.
 */
int wmibm_batch_step(wmibm_batch *b, wmibm_band_stats *stats, void *stream);

/*
 * wmibm_batch_wall_stress_force - wall stress and force of every member (the
 * step without the body mask); same launches, arguments and results otherwise.
 */
int wmibm_batch_wall_stress_force(wmibm_batch *b, wmibm_band_stats *stats, void *stream);

/*
 * wmibm_batch_device_status - reads and clears the batch's device status word,
 * which its kernels set when one of their bounded waits gave up.  Synchronises
 * `stream`.  *out receives WMIBM_OK or WMIBM_ETIMEOUT.
 */
int wmibm_batch_device_status(wmibm_batch *b, int32_t *out, void *stream);

/* Algorithmic bytes of one batch step: which = 0 wall kernel, 1 force + mask kernel. */
int64_t wmibm_batch_traffic_bytes(const wmibm_batch *b, int32_t which);

/* Total nodes of all members. */
int64_t wmibm_batch_points(const wmibm_batch *b);

const char *wmibm_batch_last_error(const wmibm_batch *b);
void wmibm_batch_destroy(wmibm_batch *b);

/* Number of entries of list `which` (WMIBM_LIST_*), or -1 for a bad argument. */
int64_t wmibm_list_size(const wmibm_handle *h, int32_t which);

/*
 * wmibm_export_list - copy list `which` (ascending int32 node indices) into the
 * HOST buffer dst of capacity cap entries; synchronises `stream`.
 * Errors: EINVAL (cap too small), ECUDA.
 */
int wmibm_export_list(wmibm_handle *h, int32_t which, int32_t *dst, int64_t cap, void *stream);

/*
 * wmibm_traffic_bytes - algorithmic bytes of one call, counted at init:
 *   which = 0: wmibm_wall_stress (band records, each distinct velocity element
 *              its stencils touch, band stress writes, the solid runs'
 *              descriptors and zero writes); 1: wmibm_force (6 stress reads + 3
 *              force writes per node); 2: wmibm_mask without grad p; 3:
 *              wmibm_mask with grad p; 4: the fused wmibm_wall_stress_force pass
 *              (force stream, band records and velocity elements, band and
 *              solid stress writes, run and row tables);
 *           5: wmibm_wall_stress's reads at the 32-byte sector granularity of
 *              the memory system: the records, every velocity sector its
 *              stencils touch, the run descriptors, and one read of every stress
 *              sector it writes (a store that does not cover its whole sector
 *              has the rest of the sector read from memory, and the stage's
 *              scattered band stores and unaligned solid runs hardly ever cover
 *              one whole);
 *           6: its writes at sector granularity: every stress sector written.
 *   Sectors are counted from element 0 of each field, i.e. for fields that
 *   start on a 32-byte boundary.
 * Returns -1 for a bad argument.
 */
int64_t wmibm_traffic_bytes(const wmibm_handle *h, int32_t which);

/* Releases everything the handle owns (waits for the device). NULL is ignored. */
void wmibm_destroy(wmibm_handle *h);

/* Static text for a status code. */
const char *wmibm_status_string(int status);

/* Text of the last error on this handle (empty if none); NULL handle: last init error. */
const char *wmibm_last_error(const wmibm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* WMIBM_H */
