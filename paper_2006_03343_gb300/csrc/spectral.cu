// The forcing f = -div(tau) with the paper's own horizontal scheme (Eq. 2 /
// Eq. 18 of Liu & Stevens, arXiv:2006.03343): x and y derivatives
// pseudo-spectral (Eqs. 13-14), vertical ones the staggered differences of
// Eqs. 15-16,
//   f_x(uv k) = -[d_x txx + d_y txy + (txz[k+1] - txz[k])/dz]
//   f_y(uv k) = -[d_x txy + d_y tyy + (tyz[k+1] - tyz[k])/dz]
//   f_z(w k)  = -[d_x txz + d_y tyz + (tzz[k] - tzz[k-1])/dz]
// with f_x = f_y = 0 on the ghost uv level and f_z = 0 on the floor and lid.
//
// The 2-D transform of Eqs. 13-14 factors by direction: multiplying the plane's
// amplitudes by i k_x touches the x index only, so d_x is the 1-D spectral
// derivative of every x-row and d_y that of every y-column.  The Nyquist bin of
// each direction carries no first derivative.  One persistent launch works
// through two kinds of unit:
//   row unit    (level k, rx rows): d_x of txx, txy, txz plus the vertical
//               terms -> writes the partial forcing into f
//   column unit (level k, wy columns): d_y of txy, tyy, tyz, subtracted from f
// Each unit stages its lines in shared memory, two real lines per complex
// sequence (z = a + i b; the derivative operator is real, so D z = D a + i D b),
// runs a radix-16/8/4/2 Stockham FFT, multiplies by i k / N while loading the first
// pass of a second forward FFT of the conjugate (IFFT(y) = conj(FFT(conj y))/N),
// and writes.  Units are dispensed by an atomic ticket in chunks of kc levels:
// the row units of chunk c, then the column units of chunk c-1.  A column unit
// on level k waits (bounded) until all row units of level k have finished, so
// the partial forcing and the stresses the two unit kinds share are re-read
// from L2 while DRAM streams each array once.  Row units never wait, and every
// row unit a column unit depends on was dispensed earlier to a running block,
// so the waits end whatever the grid size.
#include <math.h>
#include <stdlib.h>

#include "internal.cuh"
#include "tma.cuh"

namespace wmibm {

constexpr int kSpecMaxLog = 11;         // lines of up to 2048 points (FP32; 1024 for FP64)
constexpr int kSpecThreads = 256;
constexpr int kSpecBudget = 3200;       // complex elements per shared buffer aimed at (FP32; half for FP64)
constexpr double kSpecChunkBytes = 24.0 * 1024 * 1024;   // L2 footprint of one chunk of levels

struct SpecState {
    int lognx, logny;
    int rx, wy;                 // rows per row unit, columns per column unit
    int ldx, ldy;               // shared-memory stride of a sequence (complex elements, skewed and padded)
    int kc, nchunks;
    int xpl, ypl;               // units per level
    int64_t total;
    size_t smem;
    void *twx, *twy;            // omega_N^m = exp(-2 pi i m / N), m < N (dtype complex)
    void *knx, *kny;            // k_m / N per bin, Nyquist bin 0 (dtype)
    unsigned int *ctr;          // [0] ticket, [1] exit ticket, [2 + k] row units finished on level k
};

}  // namespace wmibm

using namespace wmibm;

namespace {

template <typename T>
struct Cx;
template <>
struct Cx<float> {
    using type = float2;
};
template <>
struct Cx<double> {
    using type = double2;
};

template <typename T>
struct SpecParams {
    const T *txx, *txy, *tyy, *tzz, *txz, *tyz;
    T *fx, *fy, *fz;
    const typename Cx<T>::type *twx, *twy;
    const T *knx, *kny;
    unsigned int *ctr;
    int *status;
    int32_t nx, ny, nz;
    int32_t lognx, logny, logrx, logwy;
    int32_t ldx, ldy;
    int32_t kc, nchunks, xpl, ypl;
    int64_t total;
    int32_t buf;              // complex elements per shared buffer
    int32_t v16;              // stage with 16-byte copies (every staged segment 16-byte aligned)
    T rdz;
};

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C>
__device__ __forceinline__ C cmi(C a) { return C{a.y, -a.x}; }       // -i a

// Element e of a sequence sits at e + e/32 in shared memory: the padding spreads
// the stride-R writes of the first Stockham pass over the banks.
__device__ __forceinline__ int sk(int e) { return e + (e >> 5); }

// log2 of the radix of the Stockham pass that starts at Ns = 2^logns in a
// transform of N = 2^logn points: as few passes as radix 2^maxlog allows, the
// first at the largest radix and the others as even as possible (FP32, radix up
// to 16: 256 = 16 x 16, 512 = 16 x 8 x 4, 1024 = 16 x 8 x 8; FP64, whose values
// take twice the registers: radix up to 8).  A first pass of radix 16 keeps the
// second pass's stride at Ns = 16: with the one-per-32 skew its stores spread
// two lanes to an 8-byte bank slot, where Ns = 8 (512 = 8 x 8 x 8) put four.
__host__ __device__ constexpr int pass_log(int logn, int logns, int maxlog)
{
    return logn - logns <= 0 ? 0
           : logns == 0      ? (logn < maxlog ? logn : maxlog)
                             : (logn - logns + (logn - logns + maxlog - 1) / maxlog - 1) /
                                   ((logn - logns + maxlog - 1) / maxlog);
}
template <typename T>
constexpr int kMaxPassLog = sizeof(T) == 4 ? 4 : 3;

// R-point forward DFT in registers, natural order in and out:
// V[q] = sum_r v[r] exp(-2 pi i r q / R).
template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
    template <typename C>
    __device__ __forceinline__ static void run(C *v)
    {
        const C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <typename T>
struct Dft<T, 4> {
    template <typename C>
    __device__ __forceinline__ static void run(C *v)
    {
        const C s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
        const C s1 = cadd(v[1], v[3]), d1 = cmi(csub(v[1], v[3]));
        v[0] = cadd(s0, s1);
        v[2] = csub(s0, s1);
        v[1] = cadd(d0, d1);
        v[3] = csub(d0, d1);
    }
};

template <typename T>
struct Dft<T, 16> {
    // four 4-point DFTs over the stride-4 subsequences, the twiddles
    // exp(-2 pi i r2 q1 / 16), then four 4-point DFTs across them:
    // V[q1 + 4 q2] = sum_r2 w4^(r2 q2) w16^(r2 q1) sum_r1 v[4 r1 + r2] w4^(r1 q1)
    template <typename C>
    __device__ __forceinline__ static void run(C *v)
    {
        const T c = T(0.92387953251128675613), s = T(0.38268343236508977173), h = T(0.70710678118654752440);
        C a[4][4];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
            C x[4] = {v[r2], v[4 + r2], v[8 + r2], v[12 + r2]};
            Dft<T, 4>::run(x);
#pragma unroll
            for (int q1 = 0; q1 < 4; ++q1) a[r2][q1] = x[q1];
        }
        const C w1{c, -s}, w2{h, -h}, w3{s, -c}, w6{-h, -h}, w9{-c, s};
        a[1][1] = cmul(a[1][1], w1);
        a[1][2] = cmul(a[1][2], w2);
        a[1][3] = cmul(a[1][3], w3);
        a[2][1] = cmul(a[2][1], w2);
        a[2][2] = cmi(a[2][2]);                                       // w16^4 = -i
        a[2][3] = cmul(a[2][3], w6);
        a[3][1] = cmul(a[3][1], w3);
        a[3][2] = cmul(a[3][2], w6);
        a[3][3] = cmul(a[3][3], w9);
#pragma unroll
        for (int q1 = 0; q1 < 4; ++q1) {
            C y[4] = {a[0][q1], a[1][q1], a[2][q1], a[3][q1]};
            Dft<T, 4>::run(y);
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) v[q1 + 4 * q2] = y[q2];
        }
    }
};

template <typename T>
struct Dft<T, 8> {
    // even / odd halves by two 4-point DFTs, joined with exp(-2 pi i q / 8)
    template <typename C>
    __device__ __forceinline__ static void run(C *v)
    {
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<T, 4>::run(e);
        Dft<T, 4>::run(o);
        const T h = T(0.70710678118654752440);
        o[1] = C{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};      // (1 - i)/sqrt 2
        o[2] = cmi(o[2]);                                             // -i
        o[3] = C{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};     // (-1 - i)/sqrt 2
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = cadd(e[q], o[q]);
            v[q + 4] = csub(e[q], o[q]);
        }
    }
};

// The R outputs of a first-pass butterfly (Ns = 1: element r of the butterfly at
// out[r]).  With R = 16 the elements of butterfly j start at 16 j + j/2 under the
// skew, so butterflies j and j + 1 of a half-warp share their 8-byte bank slots:
// an odd j writes its upper half first, which spreads each store's 16 lanes over
// 16 slots (FP32, NB >= 16: a half-warp holds 16 butterflies of one sequence).
template <typename T, int R, int NB, typename C>
__device__ __forceinline__ void store_first_pass(C *out, const C *v, int j)
{
    constexpr bool kRot = sizeof(T) == 4 && R == 16 && NB >= 16;
    if (kRot) {
        const bool odd = (j & 1) != 0;
        C *const lo = out + (odd ? R / 2 : 0), *const hi = out - (odd ? R / 2 : 0);
#pragma unroll
        for (int i = 0; i < R / 2; ++i) lo[i] = odd ? v[i + R / 2] : v[i];
#pragma unroll
        for (int i = R / 2; i < R; ++i) hi[i] = odd ? v[i - R / 2] : v[i];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) out[r] = v[r];
    }
}

// One Stockham pass of radix R = 2^pass_log(LOGN, LOGNS, kMaxPassLog<T>) over S sequences of length
// N = 2^LOGN, from a to b, after passes that reached Ns = 2^LOGNS.  Butterfly j
// of a sequence reads elements j + r N/R, twiddles them by
// omega_N^(r jm N/(Ns R)) with jm = j mod Ns, and writes element
// (j - jm) R + jm + r Ns.  The pass's twiddles are a table of its own,
// tw[(r - 1) Ns + jm], so that a warp's loads of one r are contiguous.  With N
// and Ns known at compile time every shared address is a base plus an
// immediate: since N/R and Ns divide 32 or are multiples of it,
// sk(j + r N/R) = sk(j) + r N/R + (r N/R)/32 and sk(o0 + r Ns) = sk(o0) + r Ns + (r Ns)/32.
// PRE: multiply each input (bin m) by i k_m / N and conjugate it first, i.e.
// v -> (-kn_m v.y, -kn_m v.x).
template <typename T, int LOGN, int LOGNS, bool PRE>
__device__ __forceinline__ void fft_pass(const typename Cx<T>::type *__restrict__ a,
                                         typename Cx<T>::type *__restrict__ b, int S, int ld,
                                         const typename Cx<T>::type *__restrict__ tw, const T *__restrict__ kn)
{
    using C = typename Cx<T>::type;
    constexpr int LOGR = pass_log(LOGN, LOGNS, kMaxPassLog<T>);
    constexpr int R = 1 << LOGR;
    constexpr int LOGNB = LOGN - LOGR;
    constexpr int NB = 1 << LOGNB;
    constexpr int NS = 1 << LOGNS;
    const int total = S << LOGNB;
    for (int t = threadIdx.x; t < total; t += kSpecThreads) {
        const int s = t >> LOGNB, j = t & (NB - 1);
        const C *in = a + s * ld + sk(j);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[r * NB + ((r * NB) >> 5)];
        if (PRE) {
            const T *k0 = kn + j;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T k = __ldg(k0 + r * NB);
                v[r] = C{-k * v[r].y, -k * v[r].x};
            }
        }
        const int jm = j & (NS - 1);
        if (LOGNS > 0) {
            const typename Cx<T>::type *w0 = tw + jm;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(w0 + (r - 1) * NS));
        }
        Dft<T, R>::run(v);
        C *out = b + s * ld + sk(((j - jm) << LOGR) + jm);
        if (LOGNS == 0) {
            store_first_pass<T, R, NB>(out, v, j);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) out[r * NS + ((r * NS) >> 5)] = v[r];
        }
    }
}

// The remaining passes of a transform, from Ns = 2^LOGNS on, ping-ponging
// between a and b with a block barrier after each; returns the buffer that holds
// the result.  tw points at the table of the pass that starts at LOGNS.
template <typename T, int LOGN, int LOGNS, bool PRE>
struct Passes {
    using C = typename Cx<T>::type;
    __device__ __forceinline__ static C *run(C *a, C *b, int S, int ld, const C *tw, const T *kn)
    {
        constexpr int LOGR = pass_log(LOGN, LOGNS, kMaxPassLog<T>);
        fft_pass<T, LOGN, LOGNS, PRE>(a, b, S, ld, tw, kn);
        __syncthreads();
        return Passes<T, LOGN, LOGNS + LOGR, false>::run(b, a, S, ld, tw + (((1 << LOGR) - 1) << LOGNS), kn);
    }
};
template <typename T, int LOGN, bool PRE>
struct Passes<T, LOGN, LOGN, PRE> {
    using C = typename Cx<T>::type;
    __device__ __forceinline__ static C *run(C *a, C *, int, int, const C *, const T *) { return a; }
};

// The first Stockham pass (Ns = 1, no twiddles) of the first transform, read
// straight from the planar staging P (planes of n = L x N values): sequence s < L
// is plane0 + i plane1 of line s, sequence L + q is plane 2 of lines 2q and 2q + 1.
// ROWS: the staging is [line][pos] and consecutive threads take consecutive
// butterflies of one sequence; otherwise it is [pos][line] and consecutive
// threads take consecutive sequences of one butterfly, so that both the staging
// reads and the skewed sequence writes stay spread over the banks.
template <typename T, int LOGN, bool ROWS>
__device__ __forceinline__ void fft_first_pass(const T *__restrict__ P, typename Cx<T>::type *__restrict__ b,
                                               int logL, int ld)
{
    using C = typename Cx<T>::type;
    constexpr int LOGR = pass_log(LOGN, 0, kMaxPassLog<T>);
    constexpr int R = 1 << LOGR;
    constexpr int LOGNB = LOGN - LOGR;
    constexpr int NB = 1 << LOGNB;
    const int L = 1 << logL;
    const int S = L + L / 2;
    const int n = L << LOGN;
    const int total = S << LOGNB;
    for (int t = threadIdx.x; t < total; t += kSpecThreads) {
        int s, j;
        if (ROWS) {
            s = t >> LOGNB;
            j = t & (NB - 1);
        } else {
            j = t / S;
            s = t - j * S;
        }
        C v[R];
        if (s < L) {
            const T *p0 = ROWS ? P + (s << LOGN) + j : P + (j << logL) + s;
            const int step = ROWS ? NB : NB << logL;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = C{p0[r * step], p0[n + r * step]};
        } else {
            const int l0 = 2 * (s - L);
            if (ROWS) {
                const T *p0 = P + 2 * n + (l0 << LOGN) + j;
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = C{p0[r * NB], p0[(1 << LOGN) + r * NB]};
            } else {
                const C *p0 = reinterpret_cast<const C *>(P + 2 * n + (j << logL) + l0);
                const int step = (NB << logL) / 2;      // complex elements between r and r + 1
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = p0[r * step];
            }
        }
        Dft<T, R>::run(v);
        C *out = b + s * ld + sk(j * R);
        if (ROWS) {
            store_first_pass<T, R, NB>(out, v, j);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) out[r] = v[r];
        }
    }
}

template <typename T, bool ROWS, int LOGN>
__device__ __forceinline__ typename Cx<T>::type *derive_n(T *P, typename Cx<T>::type *A, int logL, int ld,
                                                          const typename Cx<T>::type *tw, const T *kn)
{
    using C = typename Cx<T>::type;
    constexpr int LOGR = pass_log(LOGN, 0, kMaxPassLog<T>);
    C *B = reinterpret_cast<C *>(P);
    const int S = (1 << logL) + (1 << logL) / 2;
    fft_first_pass<T, LOGN, ROWS>(P, A, logL, ld);
    __syncthreads();
    C *r1 = Passes<T, LOGN, LOGR, false>::run(A, B, S, ld, tw + ((1 << LOGR) - 1), kn);
    return Passes<T, LOGN, 0, true>::run(r1, r1 == A ? B : A, S, ld, tw, kn);
}

// Spectral derivative of the staged lines: z = plane0 + i plane1 (and the plane-2
// pairs), conj(FFT(conj(i k/N * FFT(z)))), for N = 2^logN, 2 <= N <= 2048.  The
// first pass reads the planar staging P and writes A; P is scratch afterwards.
// The returned buffer holds (D a, -D b) for each z = a + i b.
template <typename T, bool ROWS>
__device__ __forceinline__ typename Cx<T>::type *derive(T *P, typename Cx<T>::type *A, int logL, int logN, int ld,
                                                        const typename Cx<T>::type *tw, const T *kn)
{
    switch (logN) {
    case 1: return derive_n<T, ROWS, 1>(P, A, logL, ld, tw, kn);
    case 2: return derive_n<T, ROWS, 2>(P, A, logL, ld, tw, kn);
    case 3: return derive_n<T, ROWS, 3>(P, A, logL, ld, tw, kn);
    case 4: return derive_n<T, ROWS, 4>(P, A, logL, ld, tw, kn);
    case 5: return derive_n<T, ROWS, 5>(P, A, logL, ld, tw, kn);
    case 6: return derive_n<T, ROWS, 6>(P, A, logL, ld, tw, kn);
    case 7: return derive_n<T, ROWS, 7>(P, A, logL, ld, tw, kn);
    case 8: return derive_n<T, ROWS, 8>(P, A, logL, ld, tw, kn);
    case 9: return derive_n<T, ROWS, 9>(P, A, logL, ld, tw, kn);
    case 10: return derive_n<T, ROWS, 10>(P, A, logL, ld, tw, kn);
    default: return derive_n<T, ROWS, 11>(P, A, logL, ld, tw, kn);
    }
}

// Asynchronous global -> shared copies (cp.async; completion by commit groups).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issues the copies of a unit's input lines into the planar staging buffer P:
// three planes of n = lines x line-length values (row unit: txx, txy, txz rows
// j0 .. j0 + rx - 1; column unit: txy, tyy, tyz as [ny][wy] strips), then
// commits the group (an empty group when the unit needs no input).
template <typename T, int VB>
__device__ __forceinline__ void stage_copies(const SpecParams<T> &p, T *P, int kind, int level, int idx)
{
    constexpr int V = VB / (int)sizeof(T);            // values per copy
    if (kind == 0 && level < p.nz - 1) {
        const int logn = p.logrx + p.lognx;
        const int64_t base = (int64_t)level * p.nx * p.ny + ((int64_t)idx << logn);
        const int per = (1 << logn) / V;
        for (int c = threadIdx.x; c < 3 * per; c += kSpecThreads) {
            const int f = c / per, q = c - f * per;
            const T *src = f == 0 ? p.txx : (f == 1 ? p.txy : p.txz);
            cp_async<VB>(P + ((int64_t)f << logn) + q * V, src + base + q * V);
        }
    } else if (kind == 1 && level < p.nz - 1) {
        const int logn = p.logny + p.logwy;
        const int64_t base = (int64_t)level * p.nx * p.ny + ((int64_t)idx << p.logwy);
        const int per_row = (1 << p.logwy) / V;
        const int per = per_row << p.logny;
        for (int c = threadIdx.x; c < 3 * per; c += kSpecThreads) {
            const int f = c / per, q = c - f * per;
            const int j = q / per_row, cc = q - j * per_row;
            const T *src = f == 0 ? p.txy : (f == 1 ? p.tyy : p.tyz);
            cp_async<VB>(P + ((int64_t)f << logn) + (j << p.logwy) + cc * V, src + base + (int64_t)j * p.nx + cc * V);
        }
    }
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

template <typename T>
__device__ void stage_unit(const SpecParams<T> &p, T *P, int kind, int level, int idx)
{
    if (p.v16) stage_copies<T, 16>(p, P, kind, level, idx);
    else stage_copies<T, (int)sizeof(T)>(p, P, kind, level, idx);
    cp_async_commit();
    // a row unit's epilogue reads the vertical terms of its rows (tzz at k and
    // k - 1, txz and tyz at k + 1, tyz at k), which no unit has staged yet: start
    // them towards L2 now, a unit ahead, so that the epilogue waits on L2, not DRAM
    if (kind == 0 && p.v16 && level < p.nz - 1 && threadIdx.x == 0) {
        const int64_t plane = (int64_t)p.nx * p.ny;
        const int64_t base = (int64_t)level * plane + ((int64_t)idx << (p.logrx + p.lognx));
        const uint32_t bytes = (uint32_t)(sizeof(T) << (p.logrx + p.lognx));
        prefetch_l2(p.tzz + base, bytes);
        if (level > 0) prefetch_l2(p.tzz + base - plane, bytes);
        prefetch_l2(p.tyz + base, bytes);
        prefetch_l2(p.txz + base + plane, bytes);
        prefetch_l2(p.tyz + base + plane, bytes);
    }
}

// Row unit on level k, rows j0 .. j0 + rx - 1, whose input lines are staged in
// P: d_x of txx, txy (sequences s < rx) and txz (rows 2q, 2q + 1 in rx + q),
// plus the vertical terms -> the partial forcing in f.  P is scratch afterwards.
template <typename T>
__device__ void row_unit(const SpecParams<T> &p, T *P, typename Cx<T>::type *A, int k, int j0)
{
    using C = typename Cx<T>::type;
    const int rx = 1 << p.logrx;
    const int n = rx << p.lognx;
    const int64_t plane = (int64_t)p.nx * p.ny;
    const int64_t base = (int64_t)k * plane + (int64_t)j0 * p.nx;
    if (k == p.nz - 1) {                    // ghost uv level / lid: f = 0
        for (int e = threadIdx.x; e < n; e += kSpecThreads) {
            p.fx[base + e] = T(0);
            p.fy[base + e] = T(0);
            p.fz[base + e] = T(0);
        }
        return;
    }
    const int ld = p.ldx;
    const C *R = derive<T, true>(P, A, p.logrx, p.lognx, ld, p.twx, p.knx);
#pragma unroll 4
    for (int e = threadIdx.x; e < n; e += kSpecThreads) {
        const int r = e >> p.lognx, i = e & (p.nx - 1);
        const int64_t o = base + e;
        const T xz0 = __ldg(p.txz + o), xz1 = __ldg(p.txz + o + plane);
        const T yz0 = __ldg(p.tyz + o), yz1 = __ldg(p.tyz + o + plane);
        const T zz0 = __ldg(p.tzz + o), zzm = k > 0 ? __ldg(p.tzz + o - plane) : T(0);
        const C d = R[r * ld + sk(i)];                      // (d_x txx, -d_x txy)
        const C dd = R[(rx + (r >> 1)) * ld + sk(i)];
        const T dxz = (r & 1) ? -dd.y : dd.x;               // d_x txz
        p.fx[o] = -(d.x + (xz1 - xz0) * p.rdz);
        p.fy[o] = -(-d.y + (yz1 - yz0) * p.rdz);
        p.fz[o] = (k == 0) ? T(0) : -(dxz + (zz0 - zzm) * p.rdz);
    }
}

// Waits until *ctr >= target (acquire, GPU scope); bounded by kWaitLimitNs.
__device__ bool wait_level(const unsigned int *ctr, unsigned int target, int *status)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(128);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((it & 7u) == 0) {
            if (*(volatile int *)status != 0) return false;
            if (global_timer_ns() - t0 > kWaitLimitNs) {
                atomicExch(status, kDevStatusBarrierTimeout);
                return false;
            }
        }
    }
}

// Column unit on level k, columns i0 .. i0 + wy - 1, staged in P: d_y of txy, tyy
// (sequences c < wy) and tyz (columns 2q, 2q + 1 in wy + q), subtracted from f
// once every row unit of level k has written its partial forcing.
template <typename T>
__device__ void column_unit(const SpecParams<T> &p, T *P, typename Cx<T>::type *A, int k, int i0, int *s_go)
{
    using C = typename Cx<T>::type;
    if (k == p.nz - 1) return;              // f stays 0 there (written by the row units)
    const int wy = 1 << p.logwy;
    const int n = wy << p.logny;
    const int64_t base = (int64_t)k * p.nx * p.ny + i0;
    const int ld = p.ldy;
    const C *R = derive<T, false>(P, A, p.logwy, p.logny, ld, p.twy, p.kny);
    if (threadIdx.x == 0) *s_go = wait_level(p.ctr + 2 + k, (unsigned)p.xpl, p.status) ? 1 : 0;
    __syncthreads();
    if (!*s_go) return;                     // gave up waiting: skipped, the status says so
#pragma unroll 4
    for (int e = threadIdx.x; e < n; e += kSpecThreads) {
        const int j = e >> p.logwy, c = e & (wy - 1);
        const int64_t o = base + (int64_t)j * p.nx + c;
        const T fx0 = __ldcg(p.fx + o), fy0 = __ldcg(p.fy + o), fz0 = __ldcg(p.fz + o);
        const C d = R[c * ld + sk(j)];                      // (d_y txy, -d_y tyy)
        const C dd = R[(wy + (c >> 1)) * ld + sk(j)];
        const T dyz = (c & 1) ? -dd.y : dd.x;               // d_y tyz
        p.fx[o] = fx0 - d.x;
        p.fy[o] = fy0 + d.y;
        if (k > 0) p.fz[o] = fz0 - dyz;
    }
}

// Unit u of the dispense order -> kind (0 row, 1 column), level, index within the level.
// Phase ph (0 .. nchunks): row units of chunk ph, then column units of chunk ph - 1.
template <typename T>
__device__ void decode_unit(const SpecParams<T> &p, int64_t u, int *kind, int *level, int *idx)
{
    auto start = [&](int ph) -> int64_t {
        const int64_t a = min((int64_t)ph * p.kc, (int64_t)p.nz);
        const int64_t b = min((int64_t)max(ph - 1, 0) * p.kc, (int64_t)p.nz);
        return a * p.xpl + b * p.ypl;
    };
    int lo = 0, hi = p.nchunks;             // largest ph with start(ph) <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start(mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    int64_t o = u - start(lo);
    const int64_t nrow = lo < p.nchunks ? (min((int64_t)(lo + 1) * p.kc, (int64_t)p.nz) - (int64_t)lo * p.kc) * p.xpl
                                        : 0;
    if (o < nrow) {
        *kind = 0;
        *level = lo * p.kc + (int)(o / p.xpl);
        *idx = (int)(o % p.xpl);
    } else {
        o -= nrow;
        *kind = 1;
        *level = (lo - 1) * p.kc + (int)(o / p.ypl);
        *idx = (int)(o % p.ypl);
    }
}

template <typename T>
__device__ __forceinline__ void claim(const SpecParams<T> &p, int *slot)
{
    const int64_t u = (int64_t)atomicAdd(p.ctr, 1u);
    int kind = -1, level = 0, idx = 0;
    if (u < p.total) decode_unit(p, u, &kind, &level, &idx);
    slot[0] = kind;
    slot[1] = level;
    slot[2] = idx;
}

// Persistent loop: each block holds the unit it works on and the next one, whose
// input lines stream into the other staging buffer meanwhile.  A column unit
// waits only for the row units of its level, which hold smaller tickets; the
// unfinished unit with the smallest ticket can always proceed, so the loop
// ends.  Shared memory: staging buffers P0, P1 and the FFT buffer A, each buf
// complex elements.
template <typename T>
__global__ void __launch_bounds__(kSpecThreads, sizeof(T) == 4 ? 3 : 2) k_spectral(SpecParams<T> p)
{
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char spec_smem[];
    C *A = reinterpret_cast<C *>(spec_smem);
    T *const P0 = reinterpret_cast<T *>(A + p.buf);
    T *const P1 = reinterpret_cast<T *>(A + 2 * p.buf);
    __shared__ int s_u[2][3];
    __shared__ int s_go, s_last;
    int cur = 0;
    if (threadIdx.x == 0) claim(p, s_u[0]);
    __syncthreads();
    stage_unit<T>(p, P0, s_u[0][0], s_u[0][1], s_u[0][2]);
    for (;;) {
        const int kind = s_u[cur][0], level = s_u[cur][1], idx = s_u[cur][2];
        if (kind < 0) break;
        if (threadIdx.x == 0) claim(p, s_u[cur ^ 1]);
        __syncthreads();
        stage_unit<T>(p, cur ? P0 : P1, s_u[cur ^ 1][0], s_u[cur ^ 1][1], s_u[cur ^ 1][2]);
        cp_async_wait<1>();                 // this unit's lines have landed (the next unit's may not)
        __syncthreads();
        if (kind == 0) {
            row_unit<T>(p, cur ? P1 : P0, A, level, idx << p.logrx);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(p.ctr + 2 + level, 1u);
            }
        } else {
            column_unit<T>(p, cur ? P1 : P0, A, level, idx << p.logwy, &s_go);
            __syncthreads();
        }
        cur ^= 1;
    }
    cp_async_wait<0>();
    // the last block out re-arms the counters for the next launch: every block
    // has taken its final ticket and passed its waits by then
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(p.ctr + 1, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        for (int k = threadIdx.x; k < p.nz; k += kSpecThreads) p.ctr[2 + k] = 0u;
        if (threadIdx.x == 0) p.ctr[0] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            p.ctr[1] = 0u;
        }
    }
}

int ilog2_exact(int n)
{
    if (n < 1 || (n & (n - 1))) return -1;
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

template <typename T>
int upload_tables(wmibm_handle *h, SpecState *s, cudaStream_t stream)
{
    using C = typename Cx<T>::type;
    const int n[2] = {h->nx, h->ny};
    const double len[2] = {h->lx, h->ly};
    void **tw[2] = {&s->twx, &s->twy};
    void **kn[2] = {&s->knx, &s->kny};
    for (int d = 0; d < 2; ++d) {
        const int N = n[d];
        C *ht = (C *)host_alloc(sizeof(C) * N);
        T *hk = (T *)host_alloc(sizeof(T) * N);
        if (!ht || !hk) {
            free(ht);
            free(hk);
            return set_error(nullptr, WMIBM_ENOMEM, "host memory for the spectral tables");
        }
        // per-pass twiddles: pass (Ns, R) holds omega_N^(r jm N/(Ns R)) at (r - 1) Ns + jm
        int at = 0;
        for (int logNs = 0, logN = ilog2_exact(N); logNs < logN;) {
            const int logR = pass_log(logN, logNs, kMaxPassLog<T>);
            const int Ns = 1 << logNs, R = 1 << logR;
            for (int r = 1; r < R; ++r)
                for (int jm = 0; jm < Ns; ++jm) {
                    const double a = 2.0 * M_PI * (double)r * (double)jm / (double)(Ns * R);
                    ht[at].x = (T)cos(a);
                    ht[at].y = (T)(-sin(a));
                    ++at;
                }
            logNs += logR;
        }
        for (int m = 0; m < N; ++m) {
            // wavenumber of bin m: m below N/2, m - N above, 0 for the Nyquist bin
            const int mm = (2 * m < N) ? m : (2 * m == N ? 0 : m - N);
            hk[m] = (T)(2.0 * M_PI * (double)mm / len[d] / (double)N);
        }
        cudaError_t e = dev_alloc(tw[d], sizeof(C) * N);
        if (e == cudaSuccess) e = dev_alloc(kn[d], sizeof(T) * N);
        if (e == cudaSuccess) e = cudaMemcpyAsync(*tw[d], ht, sizeof(C) * N, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(*kn[d], hk, sizeof(T) * N, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        free(ht);
        free(hk);
        if (e != cudaSuccess) return cuda_status(nullptr, e, "spectral tables");
    }
    return WMIBM_OK;
}

template <typename T>
int run_spectral(wmibm_handle *h, const SpecParams<T> &p, const SpecState *s, cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(k_spectral<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)s->smem);
    if (e != cudaSuccess) return cuda_status(h, e, "k_spectral shared memory");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spectral<T>, kSpecThreads, s->smem);
    if (e != cudaSuccess) return cuda_status(h, e, "k_spectral occupancy");
    if (per_sm < 1) return set_error(h, WMIBM_EINVAL, "spectral units do not fit on an SM");
    int64_t grid = (int64_t)per_sm * h->sm_count;
    if (grid > s->total) grid = s->total;
    k_spectral<T><<<(unsigned)grid, kSpecThreads, s->smem, stream>>>(p);
    return cuda_status(h, cudaGetLastError(), "k_spectral launch");
}

template <typename T>
int launch_spectral(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz, cudaStream_t stream)
{
    const SpecState *s = h->spec;
    SpecParams<T> p;
    p.txx = (const T *)tau[0]; p.txy = (const T *)tau[1]; p.tyy = (const T *)tau[2];
    p.tzz = (const T *)tau[3]; p.txz = (const T *)tau[4]; p.tyz = (const T *)tau[5];
    p.fx = (T *)fx; p.fy = (T *)fy; p.fz = (T *)fz;
    p.twx = (const typename Cx<T>::type *)s->twx;
    p.twy = (const typename Cx<T>::type *)s->twy;
    p.knx = (const T *)s->knx;
    p.kny = (const T *)s->kny;
    p.ctr = s->ctr;
    p.status = h->dev_status;
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz;
    p.lognx = s->lognx; p.logny = s->logny;
    p.logrx = ilog2_exact(s->rx); p.logwy = ilog2_exact(s->wy);
    p.ldx = s->ldx; p.ldy = s->ldy;
    p.kc = s->kc; p.nchunks = s->nchunks; p.xpl = s->xpl; p.ypl = s->ypl;
    p.total = s->total;
    p.buf = (int)(s->smem / (3 * sizeof(typename Cx<T>::type)));
    p.rdz = (T)(1.0 / h->dz);
    // 16-byte copies when every staged line segment starts on a 16-byte boundary
    bool v16 = (h->nx * sizeof(T)) % 16 == 0 && (s->wy * sizeof(T)) % 16 == 0;
    for (int c = 0; c < 6; ++c) v16 = v16 && ((uintptr_t)tau[c] & 15u) == 0;
    p.v16 = v16 ? 1 : 0;
    return run_spectral<T>(h, p, s, stream);
}

}  // namespace

namespace wmibm {

// Called once by wmibm_init: tables, counters and tile shapes of the spectral
// forcing when nx and ny are powers of two in [2, 2048] (FP32) or [2, 1024]
// (FP64, whose three shared buffers would not fit otherwise); otherwise the
// handle has no spectral state and wmibm_force_spectral returns WMIBM_EINVAL.
// Errors go to the thread's last error (the handle is not returned on failure).
int spectral_setup(wmibm_handle *h, cudaStream_t stream)
{
    h->spec = nullptr;
    const int lx = ilog2_exact(h->nx), ly = ilog2_exact(h->ny);
    const int maxlog = h->dtype == WMIBM_F64 ? kSpecMaxLog - 1 : kSpecMaxLog;
    if (lx < 1 || ly < 1 || lx > maxlog || ly > maxlog) return WMIBM_OK;
    SpecState *s = (SpecState *)host_alloc(sizeof(SpecState));
    if (!s) return set_error(nullptr, WMIBM_ENOMEM, "host memory for the spectral state");
    h->spec = s;
    s->lognx = lx;
    s->logny = ly;
    const bool f64 = h->dtype == WMIBM_F64;
    const size_t cs = f64 ? 16 : 8;
    const int budget = f64 ? kSpecBudget / 2 : kSpecBudget;
    // rows per row unit: even power of two dividing ny, 1.5 rx (nx + 1) within the budget
    s->ldx = h->nx + (h->nx >> 5) + 1;       // skewed sequence (e + e/32) plus one: odd-ish bank offset
    s->rx = 2;
    while (s->rx * 2 <= h->ny && 3 * (s->rx * 2) / 2 * s->ldx <= budget) s->rx *= 2;
    s->ldy = h->ny + (h->ny >> 5) + 1;
    s->wy = 2;
    while (s->wy * 2 <= h->nx && 3 * (s->wy * 2) / 2 * s->ldy <= budget) s->wy *= 2;
    const int64_t ex = (int64_t)3 * s->rx / 2 * s->ldx, ey = (int64_t)3 * s->wy / 2 * s->ldy;
    const int64_t buf = ((ex > ey ? ex : ey) + 1) & ~(int64_t)1;    // even: 16-byte aligned buffers
    s->smem = 3 * cs * (size_t)buf;
    s->xpl = h->ny / s->rx;
    s->ypl = h->nx / s->wy;
    const double level_bytes = 9.0 * (double)h->nx * (double)h->ny * (double)elem_size(h->dtype);
    s->kc = (int)(kSpecChunkBytes / level_bytes);
    if (s->kc < 1) s->kc = 1;
    if (s->kc > h->nz) s->kc = h->nz;
    s->nchunks = (h->nz + s->kc - 1) / s->kc;
    s->total = (int64_t)h->nz * (s->xpl + s->ypl);
    int st = f64 ? upload_tables<double>(h, s, stream) : upload_tables<float>(h, s, stream);
    if (st) return st;
    cudaError_t e = dev_alloc(&s->ctr, sizeof(unsigned int) * (size_t)(h->nz + 2));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ctr, 0, sizeof(unsigned int) * (size_t)(h->nz + 2), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(nullptr, e, "spectral counters");
    return WMIBM_OK;
}

void spectral_free(wmibm_handle *h)
{
    SpecState *s = h ? h->spec : nullptr;
    if (!s) return;
    if (s->twx) cudaFree(s->twx);
    if (s->twy) cudaFree(s->twy);
    if (s->knx) cudaFree(s->knx);
    if (s->kny) cudaFree(s->kny);
    if (s->ctr) cudaFree(s->ctr);
    free(s);
    h->spec = nullptr;
}

// Shape of the spectral launch, for the bench and the tests: [rows per row unit,
// columns per column unit, levels per chunk, shared bytes per block].
int spectral_shape(const wmibm_handle *h, int64_t out[4])
{
    const SpecState *s = h->spec;
    if (!s) return WMIBM_EINVAL;
    out[0] = s->rx;
    out[1] = s->wy;
    out[2] = s->kc;
    out[3] = (int64_t)s->smem;
    return WMIBM_OK;
}

}  // namespace wmibm

extern "C" int wmibm_force_spectral(wmibm_handle *h, const void *const tau[6], void *fx, void *fy, void *fz,
                                    void *stream)
{
    ApiRange nvtx_range("wmibm_force_spectral");
    if (!h) return set_error(nullptr, WMIBM_EINVAL, "NULL handle");
    if (!tau || !fx || !fy || !fz) return set_error(h, WMIBM_EINVAL, "NULL stress or force pointer");
    for (int c = 0; c < 6; ++c)
        if (!tau[c]) return set_error(h, WMIBM_EINVAL, "NULL stress pointer %d", c);
    if (!h->spec)
        return set_error(h, WMIBM_EINVAL, "spectral derivatives need nx and ny powers of two in [2, %d] (got %d x %d)",
                         h->dtype == WMIBM_F64 ? 1 << (kSpecMaxLog - 1) : 1 << kSpecMaxLog, h->nx, h->ny);
    int st = check_device(h);
    if (st) return st;
    if (h->dtype == WMIBM_F64) return launch_spectral<double>(h, tau, fx, fy, fz, (cudaStream_t)stream);
    return launch_spectral<float>(h, tau, fx, fy, fz, (cudaStream_t)stream);
}

extern "C" int wmibm_spectral_shape(const wmibm_handle *h, int64_t out[4])
{
    if (!h || !out) return WMIBM_EINVAL;
    return wmibm::spectral_shape(h, out);
}
