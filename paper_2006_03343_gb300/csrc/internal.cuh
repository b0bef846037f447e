// Internal declarations of libwmibm: the handle, the per-band-node record and
// small device helpers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>

#include "wmibm.h"

namespace wmibm {

constexpr int kThreads = 256;          // block size of the list-driven kernels
constexpr int kStatVals = 8;           // per band: sum tau_w, sum tau_w^2, min tau_w, max |U_r|

// One band node, FP32 path (48 bytes, three 16-byte vector loads).
//   nC   = (n_x, n_y, n_z, C) with C = kappa^2 / ln^2(phi_c / z0)
//   frac = (a_x, a_y, a_z on the uv-grid, a_z on the w-grid): trilinear weights
//   ix   = (node index, base corner on the uv-grid, base corner on the w-grid,
//           wrap flags: bit 0 = the +x corner wraps to i = 0, bit 1 = the +y
//           corner wraps to j = 0)
struct __align__(16) RecF32 {
    float4 nC;
    float4 frac;
    int4 ix;
};

// One band node, FP64 path (80 bytes), same fields.
struct __align__(16) RecF64 {
    double2 n01;
    double2 n2C;
    double2 fxy;
    double2 fz;
    int4 ix;
};

struct Lists {
    int32_t *p[6];
    int64_t n[6];
};

// Resolved launch shape of the pipelined stencil.
struct StencilConfig {
    int rows, stages, consumer_warps, wall_warps, blocks_per_sm;
    int wall_chunk;            // interleaved single launch: band records per wall stage (0: automatic)
    int dyn_chunk;             // units per take of the dynamic dispensing (0: a fixed share per block)
    int wall_grid;             // blocks per SM of the separate wall kernel (0: as many as fit)
};

struct SpecState;              // tables, counters and tile shapes of the spectral forcing (spectral.cu)

}  // namespace wmibm

struct wmibm_handle {
    int device;
    int32_t nx, ny, nz;
    double lx, ly, lz, dx, dy, dz;
    double phi_b, kappa, phi_c;
    int32_t dtype, vel_dtype;
    int64_t n;
    wmibm::Lists lists;
    void *rec;                  // band records: w-band first, then uv-band
    int64_t nrec;
    void *partials;             // per-block partial band statistics (dtype)
    unsigned int *ticket;       // [4] counters kept at 0 between calls (wall-kernel ticket, fused-step counters)
    double *sacc;               // [8] band-statistics accumulator, kept at 0 between calls
    int64_t partial_blocks;
    int64_t traffic[7];
    int64_t nzclamp[2];         // band nodes (w, uv) whose sample point's level was clamped
    uint64_t wait_ns;           // limit of the kernels' bounded waits (WMIBM_WAIT_LIMIT_NS at init; 1 s)
    int hold_release;           // failure-path test: the single launch never releases its dirty stages
    int2 *runs[2];              // solid runs along x (first node, length): w-grid, uv-grid
    int64_t nruns[2];
    int *dev_status;            // set by kernels whose bounded waits gave up
    int64_t occ_key[8];         // cached occupancy of stencil launch shapes
    int occ_val[8], occ_next;
    int32_t dirty_lo, dirty_hi; // stencil levels [lo, hi) whose stages read band or solid entries
    int sm_count;
    wmibm_tuning tuning;
    const void *logz0;          // per-cell ln z0 (caller-owned, dtype) set by wmibm_set_log_z0, or NULL
    // transpose of the trilinear gathers of the band records (adjoint), built once:
    int32_t *adj_keys;          // touched uv-grid nodes, then touched w-grid nodes (ascending in each)
    int32_t *adj_offs;          // [adj_m[0] + adj_m[1] + 1] offsets into adj_ent
    int32_t *adj_ent;           // record * 8 + corner (bit 0: +x, bit 1: +y, bit 2: +z)
    int64_t adj_m[2];
    void *adj_grad;             // per record: dL/du_hat (3) and dL/d(ln z0) (1), dtype
    wmibm::SpecState *spec;     // spectral forcing state, or NULL when nx or ny is not a power of two
    char err[512];
};

namespace wmibm {

// ------------------------------------------------------------------------- //
// host helpers
// ------------------------------------------------------------------------- //
int set_error(wmibm_handle *h, int status, const char *fmt, ...);
int check_device(wmibm_handle *h);
int cuda_status(wmibm_handle *h, cudaError_t e, const char *what);
int spectral_setup(wmibm_handle *h, cudaStream_t stream);     // spectral.cu, once per handle
void spectral_free(wmibm_handle *h);

inline size_t elem_size(int32_t t) { return t == WMIBM_F64 ? 8 : (t == WMIBM_BF16 ? 2 : 4); }

// An NVTX range around one entry point of the C ABI (host side: the argument
// checks and the enqueueing of its launches), named after it, so that profiler
// timelines show each call; without a profiler attached it costs a branch.
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};

// Allocations of the library go through these (fault.cu): WMIBM_FAULT=alloc:N,
// read by fault_arm() at the start of wmibm_init and wmibm_batch_create, makes
// the N-th one fail (device: cudaErrorMemoryAllocation; host: NULL).
void fault_arm();
bool fault_fires();
// Wait limit and release hold for a new handle or batch: WMIBM_WAIT_LIMIT_NS (ns,
// default 1e9, kept within [1e5, 1e10]) and WMIBM_FAULT=hold_release.
void fault_wait_settings(uint64_t *wait_ns, int *hold_release);
cudaError_t dev_alloc_bytes(void **p, size_t bytes);
void *host_alloc(size_t bytes);      // zeroed, release with free()
template <typename P>
inline cudaError_t dev_alloc(P **p, size_t bytes) { return dev_alloc_bytes(reinterpret_cast<void **>(p), bytes); }

// ------------------------------------------------------------------------- //
// device helpers
// ------------------------------------------------------------------------- //
template <typename V>
__device__ __forceinline__ float load_vel_f(const V *p, int64_t i);
template <>
__device__ __forceinline__ float load_vel_f<float>(const float *p, int64_t i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float load_vel_f<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i)
{
    return __bfloat162float(p[i]);
}

template <typename V, typename T>
__device__ __forceinline__ T load_vel(const V *p, int64_t i) { return (T)load_vel_f<V>(p, i); }
template <>
__device__ __forceinline__ double load_vel<double, double>(const double *p, int64_t i) { return __ldg(p + i); }

template <typename V, typename T>
__device__ __forceinline__ V to_vel(T x) { return (V)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_vel<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }

}  // namespace wmibm
