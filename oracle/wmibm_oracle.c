/*
 * FP64 CPU oracle of the simplified wall-modeled immersed boundary stress stage
 * of Liu & Stevens, "Wall modeled immersed boundary method for high Reynolds
 * number flow over complex terrain" (arXiv:2006.03343), Sec. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; it is
 * called only by the tests, by the package smoke check and by the CPU-baseline
 * leg of bench.py.  It shares no code, header, table or helper with the CUDA
 * path: it works straight from the level set phi at every node it visits and
 * never builds the precomputed band records the GPU path uses.
 *
 * Everything is plain double precision, plain loops, in the order the paper
 * states the steps.  Compiled with -ffp-contract=off so that no multiply-add is
 * fused behind the reader's back.
 *
 * Grid and storage (Sec. 2.4, Eq. 12 and Eqs. 15-16):
 *   dx = lx/nx, dy = ly/ny, dz = lz/(nz-1); arrays are [k][j][i], i fastest.
 *   uv-node (i,j,k) sits at (i dx, j dy, (k+1/2) dz); level k = nz-1 lies above
 *   the lid and is a ghost level.  w-node (i,j,k) sits at (i dx, j dy, k dz);
 *   k = 0 is the floor and k = nz-1 the lid.  u, v, p and the stresses
 *   txx, txy, tyy, tzz live on uv-nodes; w, txz, tyz live on w-nodes.
 *
 * Readings of the paper where it is silent:
 *   R1  phi_b is a free parameter with 2 phi_b in [dz, 1.5 dz) (Sec. 3.3);
 *       the caller passes it.
 *   R2  the velocity sample point lies at distance phi_c from the SURFACE
 *       along n: x_c = x + (phi_c - phi(x)) n (Sec. 3.3).
 *   R3  the second-order accurate interpolation = trilinear interpolation of each
 *       velocity component on its own staggered grid, periodic in x and y,
 *       clamped to the physical levels in z (uv: 0..nz-2, w: 0..nz-1).
 *   R4  grad(phi) by 2nd-order central differences on the node's own grid,
 *       periodic in x, y, one-sided at the first and last z level; a zero
 *       gradient gives n = (0,0,1).
 *   R5  the rotation tau_ij = a_im a_jn tau'_mn with only tau'_13 = tau'_31 =
 *       tau_w is carried out literally with the frame e1 = U_r/|U_r|,
 *       e2 = n x e1, e3 = n; when U_r = 0 the stress is zero.
 *   R6  horizontal derivatives of the stress divergence use 2nd-order central
 *       differences (periodic) instead of the paper's pseudo-spectral ones
 *       (Eqs. 13-14); vertical ones follow Eqs. 15-16.  f_x = f_y = 0 on the
 *       ghost uv level, f_z = 0 on the floor and lid w levels (w = 0 there,
 *       Eqs. 8 and 11).
 *   R7  a per-cell roughness z0[k][j][i] serves both the uv-node and the
 *       w-node with the same (i,j,k).
 *   R10 for terrain given as heights h[j][i] at the column nodes (i dx, j dy),
 *       the immersed boundary is the piecewise-linear surface through the
 *       samples: cell [i, i+1] x [j, j+1] is split along the diagonal from
 *       (i, j) to (i+1, j+1) into two flat triangles, periodic in x and y.
 *       phi of Sec. 3.1 is the distance d to that surface, signed by
 *       z - h[j][i] (the node's own column passes through a vertex).  Where d
 *       exceeds the caller's reach, phi keeps the vertical value z - h[j][i]
 *       (same sign, magnitude >= d > reach).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* node classes of Sec. 3.3 */
#define ORC_FLUID 0
#define ORC_BAND 1
#define ORC_SOLID 2

typedef struct {
    int64_t nx, ny, nz;
    double dx, dy, dz;
} orc_grid;

static orc_grid make_grid(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz)
{
    orc_grid g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.dx = lx / (double)nx;           /* Eq. 12 */
    g.dy = ly / (double)ny;
    g.dz = lz / (double)(nz - 1);
    return g;
}

static int64_t at(const orc_grid *g, int64_t i, int64_t j, int64_t k)
{
    return (k * g->ny + j) * g->nx + i;
}

/* periodic wrap of a horizontal index */
static int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

int orc_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of threads of the parallel loops (timing only; no effect on results). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.3: node classification.  is_w selects the w-grid rules.            */
/* ------------------------------------------------------------------------- */
static int classify_node(double phi, double phi_b, int is_w)
{
    if (is_w) {
        if (phi > phi_b) return ORC_FLUID;             /* fluid: phi > phi_b        */
        if (phi >= -phi_b) return ORC_BAND;            /* band: -phi_b <= phi <= phi_b */
        return ORC_SOLID;                              /* solid: phi < -phi_b       */
    }
    if (phi > 2.0 * phi_b) return ORC_FLUID;           /* fluid: phi > 2 phi_b      */
    if (phi >= 0.0) return ORC_BAND;                   /* band: 0 <= phi <= 2 phi_b */
    return ORC_SOLID;                                  /* solid: phi < 0            */
}

void orc_classify(int64_t nx, int64_t ny, int64_t nz, const double *phi_uv, const double *phi_w,
                  double phi_b, int8_t *cls_uv, int8_t *cls_w)
{
    int64_t n = nx * ny * nz;
    for (int64_t p = 0; p < n; ++p) {
        cls_uv[p] = (int8_t)classify_node(phi_uv[p], phi_b, 0);
        cls_w[p] = (int8_t)classify_node(phi_w[p], phi_b, 1);
    }
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: n = grad(phi) / |grad(phi)| (reading R4).                       */
/* ------------------------------------------------------------------------- */
static void normal_at(const orc_grid *g, const double *phi, int64_t i, int64_t j, int64_t k, double n[3])
{
    double gx = (phi[at(g, wrap(i + 1, g->nx), j, k)] - phi[at(g, wrap(i - 1, g->nx), j, k)]) / (2.0 * g->dx);
    double gy = (phi[at(g, i, wrap(j + 1, g->ny), k)] - phi[at(g, i, wrap(j - 1, g->ny), k)]) / (2.0 * g->dy);
    double gz;
    if (k == 0)
        gz = (phi[at(g, i, j, 1)] - phi[at(g, i, j, 0)]) / g->dz;
    else if (k == g->nz - 1)
        gz = (phi[at(g, i, j, k)] - phi[at(g, i, j, k - 1)]) / g->dz;
    else
        gz = (phi[at(g, i, j, k + 1)] - phi[at(g, i, j, k - 1)]) / (2.0 * g->dz);
    double mag = sqrt(gx * gx + gy * gy + gz * gz);
    if (mag <= 1e-12) {
        n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
        return;
    }
    n[0] = gx / mag; n[1] = gy / mag; n[2] = gz / mag;
}

void orc_normals(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                 const double *phi, double *nrm /* [3][N] */)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    int64_t n = nx * ny * nz;
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double v[3];
                normal_at(&g, phi, i, j, k, v);
                int64_t p = at(&g, i, j, k);
                nrm[p] = v[0]; nrm[n + p] = v[1]; nrm[2 * n + p] = v[2];
            }
}

/* ------------------------------------------------------------------------- */
/* Reading R3: trilinear interpolation of a field on the uv-grid (is_w = 0)  */
/* or the w-grid (is_w = 1) at the physical point (x, y, z).                 */
/* ------------------------------------------------------------------------- */
static double interp(const orc_grid *g, const double *f, int is_w, double x, double y, double z)
{
    double xi = x / g->dx;
    double eta = y / g->dy;
    double zeta = is_w ? z / g->dz : z / g->dz - 0.5;
    int64_t top = is_w ? g->nz - 1 : g->nz - 2;  /* highest physical level */
    if (zeta < 0.0) zeta = 0.0;
    if (zeta > (double)top) zeta = (double)top;

    double fi = floor(xi), fj = floor(eta), fk = floor(zeta);
    int64_t k0 = (int64_t)fk;
    if (k0 > top - 1) k0 = top - 1;
    double ax = xi - fi, ay = eta - fj, az = zeta - (double)k0;
    int64_t i0 = wrap((int64_t)fi, g->nx), i1 = wrap((int64_t)fi + 1, g->nx);
    int64_t j0 = wrap((int64_t)fj, g->ny), j1 = wrap((int64_t)fj + 1, g->ny);
    int64_t k1 = k0 + 1;

    return (1 - ax) * (1 - ay) * (1 - az) * f[at(g, i0, j0, k0)]
         + ax * (1 - ay) * (1 - az) * f[at(g, i1, j0, k0)]
         + (1 - ax) * ay * (1 - az) * f[at(g, i0, j1, k0)]
         + ax * ay * (1 - az) * f[at(g, i1, j1, k0)]
         + (1 - ax) * (1 - ay) * az * f[at(g, i0, j0, k1)]
         + ax * (1 - ay) * az * f[at(g, i1, j0, k1)]
         + (1 - ax) * ay * az * f[at(g, i0, j1, k1)]
         + ax * ay * az * f[at(g, i1, j1, k1)];
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.3: the wall model at one band node.                                */
/*   u   : velocity at distance phi_c above the surface along n (R2, R3)     */
/*   U_r = u - (u.n) n, e1 = U_r/|U_r|, e2 = n x e1, e3 = n                  */
/*   tau_w = -[kappa U_r / ln(phi_c/z0)]^2                  (Eq. 28)         */
/*   tau'_13 = tau'_31 = tau_w, all other tau'_mn = 0                        */
/*   tau_ij = a_im a_jn tau'_mn,  a_im = e_m . e_i          (rotation)       */
/* Returns the full symmetric tensor in tau[3][3] plus tau_w and |U_r|.      */
/* ------------------------------------------------------------------------- */
typedef struct {
    double tau[3][3];
    double tau_w;
    double ur;
    int zclamped;     /* 1 if x_c lies outside the physical levels of the uv-grid or the w-grid (R3) */
} orc_node_result;

static void wall_model_at(const orc_grid *g, const double *phi, int is_w,
                          int64_t i, int64_t j, int64_t k,
                          const double *u, const double *v, const double *w,
                          double lg, double phi_c, double kappa, orc_node_result *out)
{
    double n[3];
    normal_at(g, phi, i, j, k, n);

    double x = (double)i * g->dx;
    double y = (double)j * g->dy;
    double z = is_w ? (double)k * g->dz : ((double)k + 0.5) * g->dz;
    double d = phi_c - phi[at(g, i, j, k)];
    double xc = x + d * n[0], yc = y + d * n[1], zc = z + d * n[2];

    /* R3: the interpolation clamps the fractional level of z_c to the physical levels
       of each grid (uv: 0 .. nz-2, w: 0 .. nz-1, the same expressions as in interp);
       note whether it had to on either grid */
    {
        double zeta_uv = zc / g->dz - 0.5, zeta_w = zc / g->dz;
        out->zclamped = (zeta_uv < 0.0 || zeta_uv > (double)(g->nz - 2) || zeta_w < 0.0 ||
                         zeta_w > (double)(g->nz - 1)) ? 1 : 0;
    }

    double uc[3];
    uc[0] = interp(g, u, 0, xc, yc, zc);   /* u on the uv-grid */
    uc[1] = interp(g, v, 0, xc, yc, zc);   /* v on the uv-grid */
    uc[2] = interp(g, w, 1, xc, yc, zc);   /* w on the w-grid  */

    double un = uc[0] * n[0] + uc[1] * n[1] + uc[2] * n[2];
    double Ur[3] = { uc[0] - un * n[0], uc[1] - un * n[1], uc[2] - un * n[2] };
    double ur = sqrt(Ur[0] * Ur[0] + Ur[1] * Ur[1] + Ur[2] * Ur[2]);

    /* lg = ln(phi_c / z0), passed in by the caller (see roughness_log) */
    double tw = -(kappa * ur / lg) * (kappa * ur / lg);
    out->tau_w = tw;
    out->ur = ur;

    memset(out->tau, 0, sizeof(out->tau));
    if (ur == 0.0) return;                        /* R5: no tangential velocity */

    double e[3][3];                               /* e[m] = local basis vector m */
    for (int c = 0; c < 3; ++c) e[0][c] = Ur[c] / ur;
    e[1][0] = n[1] * e[0][2] - n[2] * e[0][1];    /* e2 = n x e1 */
    e[1][1] = n[2] * e[0][0] - n[0] * e[0][2];
    e[1][2] = n[0] * e[0][1] - n[1] * e[0][0];
    for (int c = 0; c < 3; ++c) e[2][c] = n[c];

    double tl[3][3] = { { 0 } };                  /* local-frame stress tau'_mn */
    tl[0][2] = tw;
    tl[2][0] = tw;

    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q)
                    s += e[m][a] * e[q][b] * tl[m][q];
            out->tau[a][b] = s;
        }
}

/*
 * ln(phi_c / z0) of node p.  z0_mode 0: z0[0] is one roughness for every node;
 * 1: z0 is a per-cell field [k][j][i] (reading R7); 2: the array holds
 * s = ln z0 per cell and the log ratio is ln(phi_c) - s (the form the adjoint
 * differentiates, C = kappa^2 / (ln phi_c - s)^2).
 */
static double roughness_log(const double *z0, int z0_mode, int64_t p, double phi_c)
{
    if (z0_mode == 2) return log(phi_c) - z0[p];
    return log(phi_c / z0[z0_mode ? p : 0]);
}

/* Kahan-compensated accumulation of the band statistics. */
typedef struct {
    int64_t count, zclamped;
    double sum_tw, c_tw, sum_tw2, c_tw2, min_tw, max_ur;
} orc_stats_acc;

static void kahan_add(double *sum, double *comp, double x)
{
    double y = x - *comp;
    double t = *sum + y;
    *comp = (t - *sum) - y;
    *sum = t;
}

static void stats_add(orc_stats_acc *s, double tw, double ur, int zclamped)
{
    s->count += 1;
    s->zclamped += zclamped;
    kahan_add(&s->sum_tw, &s->c_tw, tw);
    kahan_add(&s->sum_tw2, &s->c_tw2, tw * tw);
    if (tw < s->min_tw) s->min_tw = tw;
    if (ur > s->max_ur) s->max_ur = ur;
}

/*
 * The wall model on one grid (is_w: the w-grid, writing txz, tyz; else the
 * uv-grid, writing txx, txy, tyy, tzz), the levels shared among threads: a
 * level's band nodes are evaluated in its own loop, their (tau_w, |U_r|, clamp)
 * kept at the node's place in the grid's band order (counted per level first),
 * and the statistics added afterwards on one thread in that order, so that they
 * come out exactly as from a single loop over the nodes.  Returns 0, or -2 when
 * memory runs out.
 */
static int wall_stress_grid(const orc_grid *g, const double *phi, int is_w, double phi_b,
                            const double *z0, int z0_is_field, double phi_c, double kappa,
                            const double *u, const double *v, const double *w, double *t[4],
                            orc_stats_acc *acc)
{
    const int64_t nx = g->nx, ny = g->ny, nz = g->nz;
    int64_t *first = (int64_t *)calloc((size_t)nz + 1, sizeof(int64_t));
    if (!first) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k) {
        int64_t c = 0;
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                if (classify_node(phi[at(g, i, j, k)], phi_b, is_w) == ORC_BAND) ++c;
        first[k + 1] = c;
    }
    for (int64_t k = 0; k < nz; ++k) first[k + 1] += first[k];
    const int64_t nband = first[nz];
    double *res = (double *)malloc(sizeof(double) * 3 * (size_t)(nband > 0 ? nband : 1));
    if (!res) {
        free(first);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nz; ++k) {
        int64_t q = first[k];
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = at(g, i, j, k);
                int c = classify_node(phi[p], phi_b, is_w);
                if (c == ORC_SOLID) {
                    if (is_w) {
                        t[0][p] = 0.0; t[1][p] = 0.0;
                    } else {
                        t[0][p] = 0.0; t[1][p] = 0.0; t[2][p] = 0.0; t[3][p] = 0.0;
                    }
                } else if (c == ORC_BAND) {
                    orc_node_result r;
                    wall_model_at(g, phi, is_w, i, j, k, u, v, w, roughness_log(z0, z0_is_field, p, phi_c), phi_c,
                                  kappa, &r);
                    if (is_w) {
                        t[0][p] = r.tau[0][2];   /* txz */
                        t[1][p] = r.tau[1][2];   /* tyz */
                    } else {
                        t[0][p] = r.tau[0][0];   /* txx */
                        t[1][p] = r.tau[0][1];   /* txy */
                        t[2][p] = r.tau[1][1];   /* tyy */
                        t[3][p] = r.tau[2][2];   /* tzz */
                    }
                    res[3 * q + 0] = r.tau_w;
                    res[3 * q + 1] = r.ur;
                    res[3 * q + 2] = (double)r.zclamped;
                    ++q;
                }
            }
    }
    for (int64_t q = 0; q < nband; ++q) stats_add(acc, res[3 * q + 0], res[3 * q + 1], (int)res[3 * q + 2]);
    free(res);
    free(first);
    return 0;
}

/*
 * One wall-stress pass (Sec. 3.3).  tau arrays are in/out: fluid values pass
 * through, band values are replaced by the wall model, solid values are set
 * to zero.  txz, tyz are modeled at w-band nodes; txx, txy, tyy, tzz at
 * uv-band nodes.
 * z0: scalar (z0_is_field = 0), a per-cell field [k][j][i] (reading R7,
 * z0_is_field = 1) or a per-cell field of ln z0 (z0_is_field = 2).
 * stats (may be NULL): 2 x {count, sum tau_w, sum tau_w^2, min tau_w, max U_r,
 * nodes whose x_c was clamped in z (R3)}, first for the w-band, then for the
 * uv-band, counts stored as doubles.
 * Returns 0, -1 if some z0 does not satisfy 0 < z0 < phi_c, -2 if memory runs out.
 */
int orc_wall_stress(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                    const double *phi_uv, const double *phi_w,
                    const double *z0, int z0_is_field, double phi_c, double kappa, double phi_b,
                    const double *u, const double *v, const double *w,
                    double *txx, double *txy, double *tyy, double *tzz, double *txz, double *tyz,
                    double *stats)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    int64_t n = nx * ny * nz;
    for (int64_t p = 0; p < (z0_is_field ? n : 1); ++p) {
        double z = z0_is_field == 2 ? exp(z0[p]) : z0[p];
        if (!(z > 0.0 && z < phi_c)) return -1;
    }

    orc_stats_acc acc[2];
    memset(acc, 0, sizeof(acc));

    double *tw_[4] = { txz, tyz, NULL, NULL };              /* w-grid: txz, tyz */
    double *tuv[4] = { txx, txy, tyy, tzz };                /* uv-grid: txx, txy, tyy, tzz */
    if (wall_stress_grid(&g, phi_w, 1, phi_b, z0, z0_is_field, phi_c, kappa, u, v, w, tw_, &acc[0])) return -2;
    if (wall_stress_grid(&g, phi_uv, 0, phi_b, z0, z0_is_field, phi_c, kappa, u, v, w, tuv, &acc[1])) return -2;

    if (stats) {
        for (int s = 0; s < 2; ++s) {
            stats[6 * s + 0] = (double)acc[s].count;
            stats[6 * s + 1] = acc[s].sum_tw;
            stats[6 * s + 2] = acc[s].sum_tw2;
            stats[6 * s + 3] = acc[s].min_tw;
            stats[6 * s + 4] = acc[s].max_ur;
            stats[6 * s + 5] = (double)acc[s].zclamped;
        }
    }
    return 0;
}

/*
 * The wall model evaluated at one node only (any class), for checks of single
 * entries at sizes where a full pass is not wanted.  Writes the 3x3 tensor
 * (row major), tau_w and |U_r|.
 */
void orc_wall_model_node(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                         const double *phi, int is_w, int64_t i, int64_t j, int64_t k,
                         const double *u, const double *v, const double *w,
                         double z0, double phi_c, double kappa, double *tau9, double *tw_ur)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    orc_node_result r;
    wall_model_at(&g, phi, is_w, i, j, k, u, v, w, log(phi_c / z0), phi_c, kappa, &r);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) tau9[3 * a + b] = r.tau[a][b];
    tw_ur[0] = r.tau_w;
    tw_ur[1] = r.ur;
}

/* Reading R3 exposed for the brute-force interpolation check. */
double orc_interp(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                  const double *f, int is_w, double x, double y, double z)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    return interp(&g, f, is_w, x, y, z);
}

/* ------------------------------------------------------------------------- */
/* f = -div(tau) on the staggered grid (Eq. 2, Eq. 18; reading R6).           */
/*   f_x(uv) = -[dx txx + dy txy + (txz[k+1] - txz[k])/dz]                   */
/*   f_y(uv) = -[dx txy + dy tyy + (tyz[k+1] - tyz[k])/dz]                   */
/*   f_z(w)  = -[dx txz + dy tyz + (tzz[k] - tzz[k-1])/dz]                   */
/* ------------------------------------------------------------------------- */
void orc_force(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
               const double *txx, const double *txy, const double *tyy,
               const double *tzz, const double *txz, const double *tyz,
               double *fx, double *fy, double *fz)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = at(&g, i, j, k);
                int64_t ip = at(&g, wrap(i + 1, nx), j, k), im = at(&g, wrap(i - 1, nx), j, k);
                int64_t jp = at(&g, i, wrap(j + 1, ny), k), jm = at(&g, i, wrap(j - 1, ny), k);

                if (k == nz - 1) {            /* ghost uv level */
                    fx[p] = 0.0;
                    fy[p] = 0.0;
                } else {
                    int64_t kp = at(&g, i, j, k + 1);
                    double dtxx_dx = (txx[ip] - txx[im]) / (2.0 * g.dx);
                    double dtxy_dy = (txy[jp] - txy[jm]) / (2.0 * g.dy);
                    double dtxz_dz = (txz[kp] - txz[p]) / g.dz;                /* Eq. 16 */
                    fx[p] = -(dtxx_dx + dtxy_dy + dtxz_dz);

                    double dtxy_dx = (txy[ip] - txy[im]) / (2.0 * g.dx);
                    double dtyy_dy = (tyy[jp] - tyy[jm]) / (2.0 * g.dy);
                    double dtyz_dz = (tyz[kp] - tyz[p]) / g.dz;
                    fy[p] = -(dtxy_dx + dtyy_dy + dtyz_dz);
                }

                if (k == 0 || k == nz - 1) {  /* floor and lid: w = 0 */
                    fz[p] = 0.0;
                } else {
                    int64_t km = at(&g, i, j, k - 1);
                    double dtxz_dx = (txz[ip] - txz[im]) / (2.0 * g.dx);
                    double dtyz_dy = (tyz[jp] - tyz[jm]) / (2.0 * g.dy);
                    double dtzz_dz = (tzz[p] - tzz[km]) / g.dz;                /* Eq. 15 */
                    fz[p] = -(dtxz_dx + dtyz_dy + dtzz_dz);
                }
            }
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2, Eq. 27: u*_IB = u* where phi > 0, 3 dt/2 grad p where phi <= 0. */
/* gpx, gpy, gpz may all be NULL: then the body velocity is set to zero.      */
/* ------------------------------------------------------------------------- */
void orc_mask(int64_t nx, int64_t ny, int64_t nz, const double *phi_uv, const double *phi_w,
              double *u, double *v, double *w,
              const double *gpx, const double *gpy, const double *gpz, double dt)
{
    int64_t n = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        if (phi_uv[p] <= 0.0) {
            u[p] = gpx ? 1.5 * dt * gpx[p] : 0.0;
            v[p] = gpy ? 1.5 * dt * gpy[p] : 0.0;
        }
        if (phi_w[p] <= 0.0) {
            w[p] = gpz ? 1.5 * dt * gpz[p] : 0.0;
        }
    }
}

/* ========================================================================= */
/* Adjoint of the stage for L = sum over nodes of (gx fx + gy fy + gz fz):   */
/* the chain rule of the forward above, derived by hand and written out      */
/* step by step (no automatic differentiation).  The mask (Eq. 27) changes   */
/* the velocity after the forcing is formed, so it takes no part in dL/du.   */
/* ========================================================================= */

/*
 * Transpose of orc_force.  Every term "f[q] -= c * tau[p]" of the forward
 * becomes "gam[p] -= c * g[q]", with the loops and coefficients of orc_force,
 * term by term.  gam = dL/dtau for the six stress arrays.  Sequential: the
 * scatter would race under a parallel loop.
 */
void orc_force_adjoint(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                       const double *gx, const double *gy, const double *gz,
                       double *gxx, double *gxy, double *gyy, double *gzz, double *gxz, double *gyz)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    int64_t n = nx * ny * nz;
    for (int64_t p = 0; p < n; ++p) {
        gxx[p] = 0.0; gxy[p] = 0.0; gyy[p] = 0.0; gzz[p] = 0.0; gxz[p] = 0.0; gyz[p] = 0.0;
    }
    double hx = 1.0 / (2.0 * g.dx), hy = 1.0 / (2.0 * g.dy), hz = 1.0 / g.dz;
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = at(&g, i, j, k);
                int64_t ip = at(&g, wrap(i + 1, nx), j, k), im = at(&g, wrap(i - 1, nx), j, k);
                int64_t jp = at(&g, i, wrap(j + 1, ny), k), jm = at(&g, i, wrap(j - 1, ny), k);
                if (k < nz - 1) {
                    int64_t kp = at(&g, i, j, k + 1);
                    /* f_x[p] = -[(txx[ip] - txx[im]) hx + (txy[jp] - txy[jm]) hy + (txz[kp] - txz[p]) hz] */
                    gxx[ip] -= hx * gx[p]; gxx[im] += hx * gx[p];
                    gxy[jp] -= hy * gx[p]; gxy[jm] += hy * gx[p];
                    gxz[kp] -= hz * gx[p]; gxz[p] += hz * gx[p];
                    /* f_y[p] = -[(txy[ip] - txy[im]) hx + (tyy[jp] - tyy[jm]) hy + (tyz[kp] - tyz[p]) hz] */
                    gxy[ip] -= hx * gy[p]; gxy[im] += hx * gy[p];
                    gyy[jp] -= hy * gy[p]; gyy[jm] += hy * gy[p];
                    gyz[kp] -= hz * gy[p]; gyz[p] += hz * gy[p];
                }
                if (k > 0 && k < nz - 1) {
                    int64_t km = at(&g, i, j, k - 1);
                    /* f_z[p] = -[(txz[ip] - txz[im]) hx + (tyz[jp] - tyz[jm]) hy + (tzz[p] - tzz[km]) hz] */
                    gxz[ip] -= hx * gz[p]; gxz[im] += hx * gz[p];
                    gyz[jp] -= hy * gz[p]; gyz[jm] += hy * gz[p];
                    gzz[p] -= hz * gz[p]; gzz[km] += hz * gz[p];
                }
            }
}

/* Transpose of interp: adds a * (trilinear weight of each corner) to df. */
static void interp_adjoint(const orc_grid *g, double *df, int is_w, double x, double y, double z, double a)
{
    double xi = x / g->dx;
    double eta = y / g->dy;
    double zeta = is_w ? z / g->dz : z / g->dz - 0.5;
    int64_t top = is_w ? g->nz - 1 : g->nz - 2;
    if (zeta < 0.0) zeta = 0.0;
    if (zeta > (double)top) zeta = (double)top;

    double fi = floor(xi), fj = floor(eta), fk = floor(zeta);
    int64_t k0 = (int64_t)fk;
    if (k0 > top - 1) k0 = top - 1;
    double ax = xi - fi, ay = eta - fj, az = zeta - (double)k0;
    int64_t i0 = wrap((int64_t)fi, g->nx), i1 = wrap((int64_t)fi + 1, g->nx);
    int64_t j0 = wrap((int64_t)fj, g->ny), j1 = wrap((int64_t)fj + 1, g->ny);
    int64_t k1 = k0 + 1;

    df[at(g, i0, j0, k0)] += (1 - ax) * (1 - ay) * (1 - az) * a;
    df[at(g, i1, j0, k0)] += ax * (1 - ay) * (1 - az) * a;
    df[at(g, i0, j1, k0)] += (1 - ax) * ay * (1 - az) * a;
    df[at(g, i1, j1, k0)] += ax * ay * (1 - az) * a;
    df[at(g, i0, j0, k1)] += (1 - ax) * (1 - ay) * az * a;
    df[at(g, i1, j0, k1)] += ax * (1 - ay) * az * a;
    df[at(g, i0, j1, k1)] += (1 - ax) * ay * az * a;
    df[at(g, i1, j1, k1)] += ax * ay * az * a;
}

/*
 * Adjoint of the wall model at one band node.  With r = U_r, rho = |r| and the
 * closed form of the rotated stress (Sec. 3.3; the literal rotation above
 * equals it, which the pins check)
 *     tau_ij = -C rho (r_i n_j + n_i r_j),
 * and G the symmetric matrix with sum_ij G_ij tau_ij = sum over the node's
 * stored components of gam_c tau_c, the node's part of L is
 *     L_node = -2 C rho (r . G n).
 * With m = G n and q = r . m:
 *     dL/dr     = -2 C (q r / rho + rho m)
 *     dL/du_hat = P dL/dr,  P = I - n n^T    (r = P u_hat)
 *     dL/dC     = -2 rho q.
 * At rho = 0 the gradient is taken as zero (the stress is zero there and its
 * derivative in r tends to zero).  The velocity part is scattered to the
 * interpolation corners; returns dL/dC.
 */
static double wall_model_adjoint_at(const orc_grid *g, const double *phi, int is_w,
                                    int64_t i, int64_t j, int64_t k,
                                    const double *u, const double *v, const double *w,
                                    double lg, double phi_c, double kappa, double G[3][3],
                                    double *du, double *dv, double *dw)
{
    double n[3];
    normal_at(g, phi, i, j, k, n);

    double x = (double)i * g->dx;
    double y = (double)j * g->dy;
    double z = is_w ? (double)k * g->dz : ((double)k + 0.5) * g->dz;
    double d = phi_c - phi[at(g, i, j, k)];
    double xc = x + d * n[0], yc = y + d * n[1], zc = z + d * n[2];

    double uc[3];
    uc[0] = interp(g, u, 0, xc, yc, zc);
    uc[1] = interp(g, v, 0, xc, yc, zc);
    uc[2] = interp(g, w, 1, xc, yc, zc);

    double un = uc[0] * n[0] + uc[1] * n[1] + uc[2] * n[2];
    double r[3] = { uc[0] - un * n[0], uc[1] - un * n[1], uc[2] - un * n[2] };
    double rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (rho == 0.0) return 0.0;

    double C = (kappa / lg) * (kappa / lg);
    double m[3];
    for (int a = 0; a < 3; ++a) m[a] = G[a][0] * n[0] + G[a][1] * n[1] + G[a][2] * n[2];
    double q = r[0] * m[0] + r[1] * m[1] + r[2] * m[2];

    double dr[3];
    for (int a = 0; a < 3; ++a) dr[a] = -2.0 * C * (q * r[a] / rho + rho * m[a]);
    double nd = n[0] * dr[0] + n[1] * dr[1] + n[2] * dr[2];
    double duh[3] = { dr[0] - nd * n[0], dr[1] - nd * n[1], dr[2] - nd * n[2] };

    interp_adjoint(g, du, 0, xc, yc, zc, duh[0]);
    interp_adjoint(g, dv, 0, xc, yc, zc, duh[1]);
    interp_adjoint(g, dw, 1, xc, yc, zc, duh[2]);
    return -2.0 * rho * q;
}

/*
 * Gradients of L = sum(gx fx + gy fy + gz fz) for one stage with per-cell
 * roughness s = ln z0 (C = kappa^2 / (ln phi_c - s)^2):
 *   du, dv, dw : dL/du, dL/dv, dL/dw (u, v on the uv-grid, w on the w-grid)
 *   dlogz0     : dL/ds per cell; cell p collects its w-band node and its
 *                uv-band node (reading R7), dC/ds = 2 C / (ln phi_c - s).
 * Fluid stresses pass through and solid ones are zero, so neither depends on
 * the velocity or on s.  Returns 0, or -1 if some z0 = exp(s) is not in
 * (0, phi_c), or -2 if scratch memory cannot be had.
 */
int orc_adjoint(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                const double *phi_uv, const double *phi_w, const double *logz0,
                double phi_c, double kappa, double phi_b,
                const double *u, const double *v, const double *w,
                const double *gx, const double *gy, const double *gz,
                double *du, double *dv, double *dw, double *dlogz0)
{
    orc_grid g = make_grid(nx, ny, nz, lx, ly, lz);
    int64_t n = nx * ny * nz;
    for (int64_t p = 0; p < n; ++p) {
        double z = exp(logz0[p]);
        if (!(z > 0.0 && z < phi_c)) return -1;
    }
    double *gam = (double *)malloc(sizeof(double) * 6 * (size_t)n);
    if (!gam) return -2;
    double *gxx = gam, *gxy = gam + n, *gyy = gam + 2 * n, *gzz = gam + 3 * n, *gxz = gam + 4 * n,
           *gyz = gam + 5 * n;
    orc_force_adjoint(nx, ny, nz, lx, ly, lz, gx, gy, gz, gxx, gxy, gyy, gzz, gxz, gyz);

    for (int64_t p = 0; p < n; ++p) {
        du[p] = 0.0; dv[p] = 0.0; dw[p] = 0.0; dlogz0[p] = 0.0;
    }

    /* w-band nodes: stored components txz = tau_13, tyz = tau_23 */
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = at(&g, i, j, k);
                if (classify_node(phi_w[p], phi_b, 1) != ORC_BAND) continue;
                double G[3][3] = { { 0 } };
                G[0][2] = G[2][0] = 0.5 * gxz[p];
                G[1][2] = G[2][1] = 0.5 * gyz[p];
                double lg = roughness_log(logz0, 2, p, phi_c);
                double dC = wall_model_adjoint_at(&g, phi_w, 1, i, j, k, u, v, w, lg, phi_c, kappa, G, du, dv, dw);
                double C = (kappa / lg) * (kappa / lg);
                dlogz0[p] += dC * 2.0 * C / lg;
            }

    /* uv-band nodes: stored components txx, txy = tau_12, tyy, tzz */
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = at(&g, i, j, k);
                if (classify_node(phi_uv[p], phi_b, 0) != ORC_BAND) continue;
                double G[3][3] = { { 0 } };
                G[0][0] = gxx[p];
                G[0][1] = G[1][0] = 0.5 * gxy[p];
                G[1][1] = gyy[p];
                G[2][2] = gzz[p];
                double lg = roughness_log(logz0, 2, p, phi_c);
                double dC = wall_model_adjoint_at(&g, phi_uv, 0, i, j, k, u, v, w, lg, phi_c, kappa, G, du, dv, dw);
                double C = (kappa / lg) * (kappa / lg);
                dlogz0[p] += dC * 2.0 * C / lg;
            }
    free(gam);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact signed distance to a height field (Sec. 3.1, reading R10).            */
/* ------------------------------------------------------------------------- */

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void sub3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[0] - b[0];
    out[1] = a[1] - b[1];
    out[2] = a[2] - b[2];
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* distance from p to the segment from a to b: the nearest point is a + t (b - a)
 * with t the projection parameter clamped to [0, 1] */
static double segment_distance(const double p[3], const double a[3], const double b[3])
{
    double ab[3], ap[3], q[3];
    sub3(b, a, ab);
    sub3(p, a, ap);
    const double l2 = dot3(ab, ab);
    double t = l2 > 0.0 ? dot3(ap, ab) / l2 : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    q[0] = ap[0] - t * ab[0];
    q[1] = ap[1] - t * ab[1];
    q[2] = ap[2] - t * ab[2];
    return sqrt(dot3(q, q));
}

/* distance from p to the flat triangle (a, b, c): a triangle is convex, so the
 * nearest point is the orthogonal projection of p onto its plane when that
 * projection lies inside (then the distance is the distance to the plane), and
 * otherwise lies on one of the three edges */
static double triangle_distance(const double p[3], const double a[3], const double b[3], const double c[3])
{
    double ab[3], ac[3], n[3], ap[3];
    sub3(b, a, ab);
    sub3(c, a, ac);
    cross3(ab, ac, n);
    sub3(p, a, ap);
    const double n2 = dot3(n, n);
    if (n2 > 0.0) {
        const double s = dot3(ap, n) / n2;
        const double q[3] = {p[0] - s * n[0], p[1] - s * n[1], p[2] - s * n[2]};
        /* q is inside when it lies on the inner side of all three edges */
        const double *v[3] = {a, b, c};
        int inside = 1;
        for (int e = 0; e < 3; ++e) {
            double edge[3], vq[3], cr[3];
            sub3(v[(e + 1) % 3], v[e], edge);
            sub3(q, v[e], vq);
            cross3(edge, vq, cr);
            if (dot3(cr, n) < 0.0) inside = 0;
        }
        if (inside) return fabs(s) * sqrt(n2);
    }
    double d = segment_distance(p, a, b);
    const double d2 = segment_distance(p, b, c);
    const double d3 = segment_distance(p, c, a);
    if (d2 < d) d = d2;
    if (d3 < d) d = d3;
    return d;
}

/* Unsigned distance from each listed node to the piecewise-linear height-field
 * surface of reading R10, by brute force over every triangle of the surface.
 * The periodic image of each triangle is the one whose centroid is nearest to
 * the node (minimum image); that is the nearest image of every point of the
 * triangle whenever the distance in question is below half the period minus a
 * cell, which the caller ensures.
 *   h      : heights [ny][nx]
 *   nodes  : flat node indices (k*ny + j)*nx + i, or NULL for every node
 *   is_w   : 1 for w-nodes (z = k dz), 0 for uv-nodes (z = (k + 1/2) dz) */
void orc_heightfield_distance(int64_t nx, int64_t ny, int64_t nz, double lx, double ly, double lz,
                              const double *h, int64_t count, const int64_t *nodes, int is_w, double *dist)
{
    const orc_grid G = make_grid(nx, ny, nz, lx, ly, lz);
    const orc_grid *g = &G;
    if (!nodes) count = nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < count; ++q) {
        const int64_t idx = nodes ? nodes[q] : q;
        const int64_t i = idx % nx, j = (idx / nx) % ny, k = idx / (nx * ny);
        const double p[3] = {i * g->dx, j * g->dy, is_w ? k * g->dz : (k + 0.5) * g->dz};
        double best = INFINITY;
        for (int64_t cj = 0; cj < ny; ++cj)
            for (int64_t ci = 0; ci < nx; ++ci) {
                /* corners of cell (ci, cj) in unwrapped coordinates */
                const double x0 = ci * g->dx, x1 = (ci + 1) * g->dx;
                const double y0 = cj * g->dy, y1 = (cj + 1) * g->dy;
                const double h00 = h[cj * nx + ci], h10 = h[cj * nx + wrap(ci + 1, nx)];
                const double h01 = h[wrap(cj + 1, ny) * nx + ci];
                const double h11 = h[wrap(cj + 1, ny) * nx + wrap(ci + 1, nx)];
                const double A[3] = {x0, y0, h00}, B[3] = {x1, y0, h10};
                const double C[3] = {x1, y1, h11}, D[3] = {x0, y1, h01};
                /* the two triangles on either side of the diagonal A-C */
                const double *tri[2][3] = {{A, B, C}, {A, C, D}};
                for (int t = 0; t < 2; ++t) {
                    const double cx = (tri[t][0][0] + tri[t][1][0] + tri[t][2][0]) / 3.0;
                    const double cy = (tri[t][0][1] + tri[t][1][1] + tri[t][2][1]) / 3.0;
                    /* shift the node by whole periods to its image nearest the centroid */
                    const double sx = lx * round((p[0] - cx) / lx);
                    const double sy = ly * round((p[1] - cy) / ly);
                    const double pp[3] = {p[0] - sx, p[1] - sy, p[2]};
                    const double d = triangle_distance(pp, tri[t][0], tri[t][1], tri[t][2]);
                    if (d < best) best = d;
                }
            }
        dist[q] = best;
    }
}
