/*
 * ews_oracle.c -- plain FP64 CPU oracle of the 3D elastic velocity-stress
 * staggered-grid finite-difference scheme (arXiv 2112.15071, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded input arrays.
 *
 * The oracle is written for a reader checking it against the paper by eye:
 * one obvious loop per equation term, FP64 throughout, no blocking, fusion or
 * reordering.  OpenMP only splits the outer loop over z-planes of a pointwise
 * update (each point is computed exactly as in the serial loop).
 *
 * Passages followed (section / equation of the paper):
 *   Eq. 1 (velocity equation), Eq. 2 and Eq. 3 (stress equation and the
 *   symmetric stress tensor, isotropic stiffness from lambda, mu), Sec. 2.1.1
 *   (staggered positions), Sec. 2.1.2 Eq. 4 (4th-order staggered difference),
 *   Sec. 2.2 (in-place additive updates), Sec. 2.2.1 (medium by trilinear
 *   interpolation at staggered points), Sec. 2.2.2 (out-of-range fetches),
 *   Sec. 2.3 (velocity pass then stress pass each step), Sec. 2.4 (receivers
 *   by trilinear interpolation of the staggered velocities), Sec. 2.5
 *   (damping of outgoing waves at the edges).
 *
 * Readings where the paper is silent or garbled (each listed in the design
 * notes):
 *   R1  Eq. 4 lacks the 1/h factor; the derivative is divided by the axis
 *       spacing.
 *   R2  element [k][j][i] of each N-sized array holds its component at the
 *       staggered position of Sec. 2.1.1 relative to cell (i, j, k).
 *   R3  v lives at half steps, sigma at integer steps; the velocity pass runs
 *       first and receivers sample v^{n+1/2}.
 *   R4  medium at staggered points = linear interpolation at half offsets,
 *       i.e. arithmetic means of 2 (rho) or 4 (mu) cells; rho is averaged and
 *       then inverted; medium indices past the top edge clamp to the edge.
 *   R5  wavefield values outside the grid are zero.
 *   R6  sponge: G(d) = exp(-(alpha (W - d) / W)^2) for a cell d < W cells from
 *       a face (per axis, product over axes), applied to every field after
 *       its update, using the element's cell index.
 *   R7  C-PML (not in the paper): Komatitsch & Martin convolutional PML with
 *       kappa = 1, d = d0 q^2, alpha = pi f0 (1 - q), d0 = -3 vpmax ln(R) /
 *       (2 W h); q from the cell index; psi = b psi + a D f; D f -> D f + psi.
 *   R8  moment source: sigma_ij -= dt M_ij s_n / (dx dy dz), spread by the
 *       transposed trilinear weights on the sigma_ij grid; force source:
 *       v_i += dt b F_i s_n / (dx dy dz) on the v_i grid.
 *   R16 free surface (Sec. 2.5, vacuum formulation): cells above plane ks
 *       hold eps times lambda, mu and rho of cell (i, j, ks) below them
 *       ("low values"); the shear modulus at the xz and yz shear points on
 *       the surface plane z = ks - 1/2 is the harmonic mean of its 4 cells
 *       (the vacuum formulation's averaging; the arithmetic mean there
 *       couples light vacuum points to the rock and is unstable); a
 *       z-difference whose Eq. 4 taps (z0 +- 1/2, z0 +- 3/2) would lie on
 *       both sides of the surface plane takes the 2nd-order form
 *       (f(z0 + 1/2) - f(z0 - 1/2)) / dz instead.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C1 (9.0 / 8.0)   /* Eq. 4 inner weight */
#define ORC_C2 (-1.0 / 24.0) /* Eq. 4 outer weight */

enum { VX, VY, VZ, SXX, SYY, SZZ, SXY, SXZ, SYZ, NFIELD };
enum { BND_NONE = 0, BND_SPONGE = 1, BND_CPML = 2 };

/* Staggered offsets of each field (Sec. 2.1.1), in cells. */
static const double OFF[NFIELD][3] = {
    {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5},          /* vx vy vz     */
    {0, 0, 0},   {0, 0, 0},   {0, 0, 0},            /* sxx syy szz  */
    {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};   /* sxy sxz syz  */

typedef struct orc_sim {
    long nx, ny, nz, n;
    double h[3];
    double *f[NFIELD];
    /* effective medium at staggered points (Sec. 2.2.1, reading R4) */
    double *bx, *by, *bz;            /* buoyancy 1/rho at vx, vy, vz points */
    double *lam, *lp2m;              /* lambda, lambda + 2 mu at normal points */
    double *mxy, *mxz, *myz;         /* mu at shear points */
    double vpmax;
    /* boundary */
    int boundary, width;
    double sponge_alpha, pml_R, pml_f0, pml_dt;
    double *g[3];                    /* 1-D sponge profiles */
    double *pa[3], *pb[3];           /* 1-D C-PML coefficients */
    double *psi[18];                 /* C-PML memory variables (full size) */
    /* free surface (reading R16): first cell plane below it, -1 without */
    long fs;
    double fs_eps;
} orc_sim;

static inline long IDX(const orc_sim *s, long i, long j, long k) {
    return (k * s->ny + j) * s->nx + i;
}

/* Fetch with the zero exterior of reading R5. */
static inline double fetch(const orc_sim *s, const double *f, long i, long j, long k) {
    if (i < 0 || j < 0 || k < 0 || i >= s->nx || j >= s->ny || k >= s->nz)
        return 0.0;
    return f[IDX(s, i, j, k)];
}

/* Reading R16: does a z-difference at output position z0 (in cells) take
 * the 2nd-order form?  Yes when its outer taps z0 - 3/2 and z0 + 3/2 lie on
 * both sides of the surface plane ks - 1/2. */
static inline int second_order_z(const orc_sim *s, double z0) {
    if (s->fs < 0) return 0;
    double zs = (double)s->fs - 0.5;
    return z0 - 1.5 < zs && zs < z0 + 1.5;
}

/* Eq. 4 evaluated at a half-integer position (index + 1/2) along axis a:
 * samples at index-1, index, index+1, index+2 (positions -3/2 .. +3/2). */
static inline double d_plus(const orc_sim *s, const double *f, int a, long i, long j, long k) {
    long di = (a == 0), dj = (a == 1), dk = (a == 2);
    double fm1 = fetch(s, f, i - di, j - dj, k - dk);
    double f0 = fetch(s, f, i, j, k);
    double fp1 = fetch(s, f, i + di, j + dj, k + dk);
    double fp2 = fetch(s, f, i + 2 * di, j + 2 * dj, k + 2 * dk);
    if (a == 2 && second_order_z(s, (double)k + 0.5)) return (fp1 - f0) / s->h[a];
    return (ORC_C1 * (fp1 - f0) + ORC_C2 * (fp2 - fm1)) / s->h[a];
}

/* Eq. 4 evaluated at an integer position along axis a, for a field that is
 * staggered by +1/2 along a: samples at index-2 .. index+1. */
static inline double d_minus(const orc_sim *s, const double *f, int a, long i, long j, long k) {
    long di = (a == 0), dj = (a == 1), dk = (a == 2);
    double fm2 = fetch(s, f, i - 2 * di, j - 2 * dj, k - 2 * dk);
    double fm1 = fetch(s, f, i - di, j - dj, k - dk);
    double f0 = fetch(s, f, i, j, k);
    double fp1 = fetch(s, f, i + di, j + dj, k + dk);
    if (a == 2 && second_order_z(s, (double)k)) return (f0 - fm1) / s->h[a];
    return (ORC_C1 * (f0 - fm1) + ORC_C2 * (fp1 - fm2)) / s->h[a];
}

static long clampi(long i, long n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

static double *zalloc(long n) { return (double *)calloc((size_t)n, sizeof(double)); }

orc_sim *orc_create(long nx, long ny, long nz, double dx, double dy, double dz) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->nx = nx; s->ny = ny; s->nz = nz; s->n = nx * ny * nz;
    s->h[0] = dx; s->h[1] = dy; s->h[2] = dz;
    for (int q = 0; q < NFIELD; ++q) s->f[q] = zalloc(s->n);
    s->bx = zalloc(s->n); s->by = zalloc(s->n); s->bz = zalloc(s->n);
    s->lam = zalloc(s->n); s->lp2m = zalloc(s->n);
    s->mxy = zalloc(s->n); s->mxz = zalloc(s->n); s->myz = zalloc(s->n);
    long dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        s->g[a] = zalloc(dims[a]);
        s->pa[a] = zalloc(dims[a]);
        s->pb[a] = zalloc(dims[a]);
        for (long i = 0; i < dims[a]; ++i) s->g[a][i] = 1.0;
    }
    s->boundary = BND_NONE;
    s->fs = -1;
    return s;
}

/* Reading R16.  ks < 0: no surface.  Takes effect at the next
 * orc_set_medium, which overwrites the medium above plane ks. */
void orc_set_free_surface(orc_sim *s, long ks, double eps) {
    s->fs = ks;
    s->fs_eps = eps;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    for (int q = 0; q < NFIELD; ++q) free(s->f[q]);
    free(s->bx); free(s->by); free(s->bz); free(s->lam); free(s->lp2m);
    free(s->mxy); free(s->mxz); free(s->myz);
    for (int a = 0; a < 3; ++a) { free(s->g[a]); free(s->pa[a]); free(s->pb[a]); }
    for (int p = 0; p < 18; ++p) free(s->psi[p]);
    free(s);
}

/* Effective medium at the staggered points (Sec. 2.2.1, reading R4).
 * Input: Lame parameters and density per cell, [nz][ny][nx]. */
void orc_set_medium(orc_sim *s, const double *lam_in, const double *mu_in,
                    const double *rho_in) {
    long nx = s->nx, ny = s->ny, nz = s->nz;
    double vpmax = 0.0;
    /* vacuum above a free surface (reading R16): eps times the column's
     * medium at plane ks */
    double *lam = zalloc(s->n), *mu = zalloc(s->n), *rho = zalloc(s->n);
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                if (s->fs >= 0 && k < s->fs) {
                    long b = IDX(s, i, j, s->fs);
                    lam[c] = s->fs_eps * lam_in[b];
                    mu[c] = s->fs_eps * mu_in[b];
                    rho[c] = s->fs_eps * rho_in[b];
                } else {
                    lam[c] = lam_in[c];
                    mu[c] = mu_in[c];
                    rho[c] = rho_in[c];
                }
            }
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                long ip = clampi(i + 1, nx), jp = clampi(j + 1, ny), kp = clampi(k + 1, nz);
                /* rho at vx (i+1/2, j, k), vy (i, j+1/2, k), vz (i, j, k+1/2) */
                s->bx[c] = 1.0 / (0.5 * (rho[c] + rho[IDX(s, ip, j, k)]));
                s->by[c] = 1.0 / (0.5 * (rho[c] + rho[IDX(s, i, jp, k)]));
                s->bz[c] = 1.0 / (0.5 * (rho[c] + rho[IDX(s, i, j, kp)]));
                s->lam[c] = lam[c];
                s->lp2m[c] = lam[c] + 2.0 * mu[c];
                /* mu at sxy (i+1/2, j+1/2, k), sxz (i+1/2, j, k+1/2), syz (i, j+1/2, k+1/2) */
                s->mxy[c] = 0.25 * (mu[c] + mu[IDX(s, ip, j, k)] + mu[IDX(s, i, jp, k)]
                                    + mu[IDX(s, ip, jp, k)]);
                s->mxz[c] = 0.25 * (mu[c] + mu[IDX(s, ip, j, k)] + mu[IDX(s, i, j, kp)]
                                    + mu[IDX(s, ip, j, kp)]);
                s->myz[c] = 0.25 * (mu[c] + mu[IDX(s, i, jp, k)] + mu[IDX(s, i, j, kp)]
                                    + mu[IDX(s, i, jp, kp)]);
                if (s->fs >= 1 && k == s->fs - 1) {
                    /* shear points on the surface plane (reading R16):
                     * harmonic mean of the 4 cells around them */
                    s->mxz[c] = 4.0 / (1.0 / mu[c] + 1.0 / mu[IDX(s, ip, j, k)]
                                       + 1.0 / mu[IDX(s, i, j, kp)] + 1.0 / mu[IDX(s, ip, j, kp)]);
                    s->myz[c] = 4.0 / (1.0 / mu[c] + 1.0 / mu[IDX(s, i, jp, k)]
                                       + 1.0 / mu[IDX(s, i, j, kp)] + 1.0 / mu[IDX(s, i, jp, kp)]);
                }
                double vp = sqrt((lam[c] + 2.0 * mu[c]) / rho[c]);
                if (vp > vpmax) vpmax = vp;
            }
    s->vpmax = vpmax;
    free(lam); free(mu); free(rho);
}

double orc_vpmax(const orc_sim *s) { return s->vpmax; }

/* Reading R17 (Sec. 2.2.1: the medium textures may be much smaller than
 * the wavefield textures and are sampled with trilinear interpolation): a
 * medium grid of m = (mx, my, mz) cells covers the same box as the n cells
 * of the wavefield grid.  A fine-grid position x (in cells, per axis) maps
 * to the medium coordinate c = (x + 1/2) m / n - 1/2 (texel centres of both
 * grids at their cell centres), clamped to [0, m - 1]; the value there is
 * the linear interpolation of the two neighbouring medium cells, per axis.
 * With m = n this is reading R4 (means of 2 or 4 cells, top edge clamped). */
static double coarse_at(const double *a, const long m[3], const long n[3], const double x[3]) {
    long i0[3];
    double fr[3];
    for (int d = 0; d < 3; ++d) {
        double c = (x[d] + 0.5) * (double)m[d] / (double)n[d] - 0.5;
        if (c < 0.0) c = 0.0;
        if (c > (double)(m[d] - 1)) c = (double)(m[d] - 1);
        i0[d] = (long)floor(c);
        if (i0[d] > m[d] - 2) i0[d] = m[d] - 2 < 0 ? 0 : m[d] - 2;
        fr[d] = c - (double)i0[d];
    }
    double v = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1])
                           * (dz ? fr[2] : 1.0 - fr[2]);
                if (w == 0.0) continue;
                long ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
                v += w * a[(iz * m[1] + iy) * m[0] + ix];
            }
    return v;
}

/* Effective medium of the staggered points from a medium grid of mx x my x
 * mz cells (reading R17): 1 / rho at the v points, lambda and lambda + 2 mu
 * at the normal points, mu at the shear points, each interpolated at its
 * own position.  vp_max is taken over the medium cells (an upper bound of
 * the interpolated speeds).  No free surface. */
void orc_set_medium_coarse(orc_sim *s, long mx, long my, long mz, const double *lam,
                           const double *mu, const double *rho) {
    const long m[3] = {mx, my, mz}, n[3] = {s->nx, s->ny, s->nz};
    double vpmax = 0.0;
    for (long c = 0; c < mx * my * mz; ++c) {
        double vp = sqrt((lam[c] + 2.0 * mu[c]) / rho[c]);
        if (vp > vpmax) vpmax = vp;
    }
    for (long k = 0; k < s->nz; ++k)
        for (long j = 0; j < s->ny; ++j)
            for (long i = 0; i < s->nx; ++i) {
                long c = IDX(s, i, j, k);
                double I = (double)i, J = (double)j, K = (double)k;
                double px[3] = {I + 0.5, J, K}, py[3] = {I, J + 0.5, K}, pz[3] = {I, J, K + 0.5};
                double p0[3] = {I, J, K};
                double pxy[3] = {I + 0.5, J + 0.5, K}, pxz[3] = {I + 0.5, J, K + 0.5};
                double pyz[3] = {I, J + 0.5, K + 0.5};
                s->bx[c] = 1.0 / coarse_at(rho, m, n, px);
                s->by[c] = 1.0 / coarse_at(rho, m, n, py);
                s->bz[c] = 1.0 / coarse_at(rho, m, n, pz);
                s->lam[c] = coarse_at(lam, m, n, p0);
                s->lp2m[c] = s->lam[c] + 2.0 * coarse_at(mu, m, n, p0);
                s->mxy[c] = coarse_at(mu, m, n, pxy);
                s->mxz[c] = coarse_at(mu, m, n, pxz);
                s->myz[c] = coarse_at(mu, m, n, pyz);
            }
    s->vpmax = vpmax;
}

/* Damping layers (Sec. 2.5 for the sponge; C-PML is reading R7).
 * Must be called after orc_set_medium (C-PML uses vpmax) and whenever dt
 * changes (C-PML coefficients depend on dt). */
void orc_set_boundary(orc_sim *s, int kind, int width, double sponge_alpha,
                      double pml_R, double pml_f0, double dt) {
    long dims[3] = {s->nx, s->ny, s->nz};
    s->boundary = kind; s->width = width;
    s->sponge_alpha = sponge_alpha; s->pml_R = pml_R; s->pml_f0 = pml_f0; s->pml_dt = dt;
    for (int a = 0; a < 3; ++a) {
        long n = dims[a];
        for (long i = 0; i < n; ++i) {
            s->g[a][i] = 1.0; s->pa[a][i] = 0.0; s->pb[a][i] = 0.0;
            long d = i < n - 1 - i ? i : n - 1 - i;       /* cells from the face */
            if (kind == BND_SPONGE && d < width) {
                double x = sponge_alpha * (double)(width - d) / (double)width;
                s->g[a][i] = exp(-x * x);
            }
            if (kind == BND_CPML && (i < width || i >= n - width)) {
                double q = i < width ? (double)(width - i) / width
                                     : (double)(i - (n - 1 - width)) / width;
                double L = width * s->h[a];
                double d0 = -3.0 * s->vpmax * log(pml_R) / (2.0 * L);
                double dd = d0 * q * q;
                double al = M_PI * pml_f0 * (1.0 - q);
                double b = exp(-(dd + al) * dt);
                s->pb[a][i] = b;
                s->pa[a][i] = (dd + al) > 0.0 ? dd * (b - 1.0) / (dd + al) : 0.0;
            }
        }
    }
    for (int p = 0; p < 18; ++p) {
        free(s->psi[p]);
        s->psi[p] = kind == BND_CPML ? zalloc(s->n) : NULL;
    }
}

/* C-PML correction of one derivative term (reading R7): inside the slab of
 * the derivative's axis the memory variable is advanced and added. */
static inline double pml_term(orc_sim *s, int p, int a, long ia, long c, double d) {
    long dims[3] = {s->nx, s->ny, s->nz};
    if (s->boundary != BND_CPML) return d;
    if (!(ia < s->width || ia >= dims[a] - s->width)) return d;
    double *psi = s->psi[p];
    psi[c] = s->pb[a][ia] * psi[c] + s->pa[a][ia] * d;
    return d + psi[c];
}

static void apply_sponge(orc_sim *s, int f0, int f1) {
    if (s->boundary != BND_SPONGE) return;
    long nx = s->nx, ny = s->ny, nz = s->nz;
    #pragma omp parallel for
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double gg = s->g[0][i] * s->g[1][j] * s->g[2][k];
                for (int q = f0; q < f1; ++q) s->f[q][IDX(s, i, j, k)] *= gg;
            }
}

/* Velocity pass, Eq. 1 with Eq. 4 (no source, no sponge):
 *   v_i += dt * b_i * sum_j D_j sigma_ij. */
static void velocity_update(orc_sim *s, double dt) {
    double **f = s->f;
    long nx = s->nx, ny = s->ny, nz = s->nz;
    #pragma omp parallel for
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                /* vx at (i+1/2, j, k) */
                double dxx = pml_term(s, 0, 0, i, c, d_plus(s, f[SXX], 0, i, j, k));
                double dxy = pml_term(s, 1, 1, j, c, d_minus(s, f[SXY], 1, i, j, k));
                double dxz = pml_term(s, 2, 2, k, c, d_minus(s, f[SXZ], 2, i, j, k));
                /* vy at (i, j+1/2, k) */
                double dyx = pml_term(s, 3, 0, i, c, d_minus(s, f[SXY], 0, i, j, k));
                double dyy = pml_term(s, 4, 1, j, c, d_plus(s, f[SYY], 1, i, j, k));
                double dyz = pml_term(s, 5, 2, k, c, d_minus(s, f[SYZ], 2, i, j, k));
                /* vz at (i, j, k+1/2) */
                double dzx = pml_term(s, 6, 0, i, c, d_minus(s, f[SXZ], 0, i, j, k));
                double dzy = pml_term(s, 7, 1, j, c, d_minus(s, f[SYZ], 1, i, j, k));
                double dzz = pml_term(s, 8, 2, k, c, d_plus(s, f[SZZ], 2, i, j, k));
                f[VX][c] += dt * s->bx[c] * (dxx + dxy + dxz);
                f[VY][c] += dt * s->by[c] * (dyx + dyy + dyz);
                f[VZ][c] += dt * s->bz[c] * (dzx + dzy + dzz);
            }
}

/* Stress pass, Eq. 2/3 with Eq. 4 (no source, no sponge):
 *   sigma_ii += dt [(lam + 2 mu) e_ii + lam (e_jj + e_kk)],
 *   sigma_ij += dt mu (D_j v_i + D_i v_j). */
static void stress_update(orc_sim *s, double dt) {
    double **f = s->f;
    long nx = s->nx, ny = s->ny, nz = s->nz;
    #pragma omp parallel for
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                double exx = pml_term(s, 9, 0, i, c, d_minus(s, f[VX], 0, i, j, k));
                double eyy = pml_term(s, 10, 1, j, c, d_minus(s, f[VY], 1, i, j, k));
                double ezz = pml_term(s, 11, 2, k, c, d_minus(s, f[VZ], 2, i, j, k));
                double vxy = pml_term(s, 12, 1, j, c, d_plus(s, f[VX], 1, i, j, k));
                double vyx = pml_term(s, 13, 0, i, c, d_plus(s, f[VY], 0, i, j, k));
                double vxz = pml_term(s, 14, 2, k, c, d_plus(s, f[VX], 2, i, j, k));
                double vzx = pml_term(s, 15, 0, i, c, d_plus(s, f[VZ], 0, i, j, k));
                double vyz = pml_term(s, 16, 2, k, c, d_plus(s, f[VY], 2, i, j, k));
                double vzy = pml_term(s, 17, 1, j, c, d_plus(s, f[VZ], 1, i, j, k));
                double l = s->lam[c], l2m = s->lp2m[c];
                f[SXX][c] += dt * (l2m * exx + l * (eyy + ezz));
                f[SYY][c] += dt * (l2m * eyy + l * (exx + ezz));
                f[SZZ][c] += dt * (l2m * ezz + l * (exx + eyy));
                f[SXY][c] += dt * s->mxy[c] * (vxy + vyx);
                f[SXZ][c] += dt * s->mxz[c] * (vxz + vzx);
                f[SYZ][c] += dt * s->myz[c] * (vyz + vzy);
            }
}

/* Trilinear weights of a point on the grid of field q (Sec. 2.4): the 8
 * neighbouring elements and their weights.  Returns 0 if any neighbour with a
 * nonzero weight falls outside the grid. */
static int trilinear(const orc_sim *s, int q, const double pos[3], long idx[8], double w[8]) {
    long dims[3] = {s->nx, s->ny, s->nz};
    long i0[3]; double fr[3];
    for (int a = 0; a < 3; ++a) {
        double u = pos[a] / s->h[a] - OFF[q][a];
        double fl = floor(u);
        i0[a] = (long)fl; fr[a] = u - fl;
    }
    int m = 0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di, ++m) {
                double wx = di ? fr[0] : 1.0 - fr[0];
                double wy = dj ? fr[1] : 1.0 - fr[1];
                double wz = dk ? fr[2] : 1.0 - fr[2];
                long ii = i0[0] + di, jj = i0[1] + dj, kk = i0[2] + dk;
                w[m] = wx * wy * wz;
                if (ii < 0 || jj < 0 || kk < 0 || ii >= dims[0] || jj >= dims[1] || kk >= dims[2]) {
                    if (w[m] != 0.0) return 0;
                    idx[m] = -1;
                } else {
                    idx[m] = IDX(s, ii, jj, kk);
                }
            }
    return 1;
}

/* Force source into the velocity pass (reading R8). */
static int inject_force(orc_sim *s, double dt, const double pos[3], const double F[3], double amp) {
    double vol = s->h[0] * s->h[1] * s->h[2];
    const double *b[3] = {s->bx, s->by, s->bz};
    for (int q = 0; q < 3; ++q) {
        long idx[8]; double w[8];
        if (!trilinear(s, q, pos, idx, w)) return 0;
        for (int m = 0; m < 8; ++m)
            if (idx[m] >= 0) s->f[q][idx[m]] += w[m] * dt * b[q][idx[m]] * F[q] * amp / vol;
    }
    return 1;
}

/* Moment-rate source into the stress pass (reading R8); M = (xx, yy, zz, xy, xz, yz). */
static int inject_moment(orc_sim *s, double dt, const double pos[3], const double M[6], double amp) {
    double vol = s->h[0] * s->h[1] * s->h[2];
    for (int c = 0; c < 6; ++c) {
        int q = SXX + c;
        long idx[8]; double w[8];
        if (!trilinear(s, q, pos, idx, w)) return 0;
        for (int m = 0; m < 8; ++m)
            if (idx[m] >= 0) s->f[q][idx[m]] -= w[m] * dt * M[c] * amp / vol;
    }
    return 1;
}

/* One velocity pass with optional force (kind 1) and the sponge. */
int orc_step_velocity(orc_sim *s, double dt, int src_kind, const double *pos,
                      const double *comp, double amp) {
    velocity_update(s, dt);
    if (src_kind == 1 && !inject_force(s, dt, pos, comp, amp)) return -1;
    apply_sponge(s, VX, VZ + 1);
    return 0;
}

/* One stress pass with optional moment source (kind 0) and the sponge. */
int orc_step_stress(orc_sim *s, double dt, int src_kind, const double *pos,
                    const double *comp, double amp) {
    stress_update(s, dt);
    if (src_kind == 0 && !inject_moment(s, dt, pos, comp, amp)) return -1;
    apply_sponge(s, SXX, SYZ + 1);
    return 0;
}

/* Trilinear sample of vx, vy, vz at each receiver (Sec. 2.4).
 * out[c * nrec + r] for component c. */
int orc_sample(const orc_sim *s, int nrec, const double *rpos, double *out) {
    for (int r = 0; r < nrec; ++r)
        for (int q = 0; q < 3; ++q) {
            long idx[8]; double w[8];
            if (!trilinear(s, q, rpos + 3 * r, idx, w)) return -1;
            double acc = 0.0;
            for (int m = 0; m < 8; ++m)
                if (idx[m] >= 0) acc += w[m] * s->f[q][idx[m]];
            out[q * nrec + r] = acc;
        }
    return 0;
}

/* The time loop (Sec. 2.3, reading R3): for n = 0 .. nt-1
 *   velocity pass (+ force s_n) -> sponge -> receivers record v^{n+1/2}
 *   stress pass (- moment s_n)  -> sponge.
 * seis is [3][nrec][nt].  snap (optional) receives every field of
 * snap_mask each snap_every steps after the stress pass, [nsnap][nmask][N]. */
int orc_forward(orc_sim *s, int nt, double dt, int src_kind, const double *pos,
                const double *comp, const double *wavelet, int nrec, const double *rpos,
                double *seis, int snap_every, unsigned snap_mask, double *snap) {
    double *tmp = (double *)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
    long isnap = 0;
    for (int n = 0; n < nt; ++n) {
        if (orc_step_velocity(s, dt, src_kind, pos, comp, wavelet[n]) != 0) { free(tmp); return -1; }
        if (nrec > 0) {
            if (orc_sample(s, nrec, rpos, tmp) != 0) { free(tmp); return -2; }
            for (int q = 0; q < 3; ++q)
                for (int r = 0; r < nrec; ++r)
                    seis[((long)q * nrec + r) * nt + n] = tmp[q * nrec + r];
        }
        if (orc_step_stress(s, dt, src_kind, pos, comp, wavelet[n]) != 0) { free(tmp); return -1; }
        if (snap && snap_every > 0 && (n + 1) % snap_every == 0) {
            for (int q = 0; q < NFIELD; ++q)
                if (snap_mask & (1u << q)) {
                    memcpy(snap + isnap * s->n, s->f[q], sizeof(double) * s->n);
                    ++isnap;
                }
        }
    }
    free(tmp);
    return 0;
}

/* Wavefield state access: state is [9][N] in field order vx vy vz sxx syy szz sxy sxz syz. */
void orc_get_state(const orc_sim *s, double *out) {
    for (int q = 0; q < NFIELD; ++q) memcpy(out + q * s->n, s->f[q], sizeof(double) * s->n);
}
void orc_set_state(orc_sim *s, const double *in) {
    for (int q = 0; q < NFIELD; ++q) memcpy(s->f[q], in + q * s->n, sizeof(double) * s->n);
    for (int p = 0; p < 18; ++p)
        if (s->psi[p]) memset(s->psi[p], 0, sizeof(double) * s->n);
}
/* C-PML memory variables, [18][N] (zeros outside the slabs). */
int orc_get_psi(const orc_sim *s, double *out) {
    if (s->boundary != BND_CPML) return -1;
    for (int p = 0; p < 18; ++p) memcpy(out + p * s->n, s->psi[p], sizeof(double) * s->n);
    return 0;
}

/* Effective-medium arrays, [8][N]: bx by bz lam lp2m mxy mxz myz. */
void orc_get_medium(const orc_sim *s, double *out) {
    const double *m[8] = {s->bx, s->by, s->bz, s->lam, s->lp2m, s->mxy, s->mxz, s->myz};
    for (int q = 0; q < 8; ++q) memcpy(out + q * s->n, m[q], sizeof(double) * s->n);
}

/* Discrete energy of the leapfrog scheme (boundaries off, no source):
 *   E^n = 1/2 sum rho_v v^{n-1/2} v^{n+1/2} + 1/2 sum sigma^n : C^{-1} : sigma^n,
 * times the cell volume.  vprev = v^{n-1/2} as [3][N]; the current state
 * holds v^{n+1/2} and sigma^n. */
double orc_energy(const orc_sim *s, const double *vprev) {
    double kin = 0.0, pot = 0.0;
    const double *b[3] = {s->bx, s->by, s->bz};
    for (int q = 0; q < 3; ++q)
        for (long c = 0; c < s->n; ++c)
            kin += vprev[q * s->n + c] * s->f[q][c] / b[q][c];
    for (long c = 0; c < s->n; ++c) {
        double l = s->lam[c], mu = 0.5 * (s->lp2m[c] - l);
        double sxx = s->f[SXX][c], syy = s->f[SYY][c], szz = s->f[SZZ][c];
        double tr = sxx + syy + szz;
        /* isotropic compliance: e = (sigma - lam / (3 lam + 2 mu) tr I) / (2 mu) */
        double enorm = (sxx * sxx + syy * syy + szz * szz
                        - l / (3.0 * l + 2.0 * mu) * tr * tr) / (2.0 * mu);
        pot += enorm;
        pot += s->f[SXY][c] * s->f[SXY][c] / s->mxy[c];
        pot += s->f[SXZ][c] * s->f[SXZ][c] / s->mxz[c];
        pot += s->f[SYZ][c] * s->f[SYZ][c] / s->myz[c];
    }
    return 0.5 * (kin + pot) * s->h[0] * s->h[1] * s->h[2];
}

/* ------------------------------------------------------------------------
 * Adjoint of the time loop (reverse mode of the discrete scheme; not in the
 * paper -- it differentiates Eq. 1-4 as discretised above).
 *
 * For a functional L of the seismograms with dL/dseis = sadj ([3][nrec][nt]),
 * returns dL/dlambda, dL/dmu, dL/drho per cell.  Boundary: none or sponge
 * (the sponge gain is diagonal, so its transpose is itself).  The forward
 * step n is
 *     V: v' = G (v + dt B Dsig(sigma) + f_n),   R: s_n = S v',
 *     T: sigma' = G (sigma + dt C Dv(v') - m_n).
 * Going back through T then V:
 *     w = G a_sig;  g_C += dt Dv(v') (x) w;  a_v += dt Dv^T(C w) + S^T sadj_n;
 *     a_sig = w;  u = G a_v;  g_B += (dt Dsig(sigma) + f_n / B) (x) u;
 *     a_sig += dt Dsig^T(B u);  a_v = u.
 * The transposes are taken column by column from the differences' own
 * weights (grad_q_T, div_tau_T), so they hold with the free-surface switch
 * of R16 too; with the zero exterior alone Dv^T = -Dsig.  The medium chain
 * rule follows the means of R4 (harmonic on the surface plane, R16) and
 * folds the vacuum cells into the surface cell of their column.
 * The forward states of each segment are recomputed from checkpoints.
 * ------------------------------------------------------------------------ */

/* velocity-pass derivative terms of an arbitrary 6-component stress-like
 * field tau (order sxx syy szz sxy sxz syz) at (i, j, k), no buoyancy. */
static void div_tau(const orc_sim *s, double *const tau[6], long i, long j, long k, double out[3]) {
    out[0] = d_plus(s, tau[0], 0, i, j, k) + d_minus(s, tau[3], 1, i, j, k) + d_minus(s, tau[4], 2, i, j, k);
    out[1] = d_minus(s, tau[3], 0, i, j, k) + d_plus(s, tau[1], 1, i, j, k) + d_minus(s, tau[5], 2, i, j, k);
    out[2] = d_minus(s, tau[4], 0, i, j, k) + d_minus(s, tau[5], 1, i, j, k) + d_plus(s, tau[2], 2, i, j, k);
}

/* stress-pass strain-rate terms of an arbitrary 3-component velocity-like
 * field q at (i, j, k): (exx, eyy, ezz, gxy, gxz, gyz). */
static void grad_q(const orc_sim *s, double *const q[3], long i, long j, long k, double e[6]) {
    e[0] = d_minus(s, q[0], 0, i, j, k);
    e[1] = d_minus(s, q[1], 1, i, j, k);
    e[2] = d_minus(s, q[2], 2, i, j, k);
    e[3] = d_plus(s, q[0], 1, i, j, k) + d_plus(s, q[1], 0, i, j, k);
    e[4] = d_plus(s, q[0], 2, i, j, k) + d_plus(s, q[2], 0, i, j, k);
    e[5] = d_plus(s, q[1], 2, i, j, k) + d_plus(s, q[2], 1, i, j, k);
}

/* Weight of the sample at offset d (cells along axis a) in the difference
 * at output index o: d_plus (output at o + 1/2) samples o-1 .. o+2,
 * d_minus (output at o) samples o-2 .. o+1; Eq. 4 weights, or the 2nd-order
 * pair where reading R16 switches the z-difference. */
static double tap_weight(const orc_sim *s, int a, int plus, long o, long d) {
    int second = a == 2 && second_order_z(s, plus ? (double)o + 0.5 : (double)o);
    long in0 = plus ? 0 : -1;             /* the inner samples are in0, in0 + 1 */
    double w = 0.0;
    if (d == in0) w = second ? -1.0 : -ORC_C1;
    else if (d == in0 + 1) w = second ? 1.0 : ORC_C1;
    else if (d == in0 - 1) w = second ? 0.0 : -ORC_C2;
    else if (d == in0 + 2) w = second ? 0.0 : ORC_C2;
    return w / s->h[a];
}

/* Transpose of d_plus (plus = 1) or d_minus (plus = 0) along axis a,
 * applied to y and evaluated at element (i, j, k): the sum over the outputs
 * o along a whose samples include the element, of that sample's weight
 * times y at o (column (i, j, k) of the difference operator). */
static double d_transpose(const orc_sim *s, const double *y, int a, int plus, long i, long j,
                          long k) {
    long dims[3] = {s->nx, s->ny, s->nz};
    long p = a == 0 ? i : (a == 1 ? j : k);
    double acc = 0.0;
    for (long o = p - 2; o <= p + 2; ++o) {
        if (o < 0 || o >= dims[a]) continue;
        double w = tap_weight(s, a, plus, o, p - o);
        if (w == 0.0) continue;
        long oi = a == 0 ? o : i, oj = a == 1 ? o : j, ok = a == 2 ? o : k;
        acc += w * y[IDX(s, oi, oj, ok)];
    }
    return acc;
}

/* Transpose of grad_q: 6 strain-like components y -> 3 velocity-like. */
static void grad_q_T(const orc_sim *s, double *const y[6], long i, long j, long k, double out[3]) {
    out[0] = d_transpose(s, y[0], 0, 0, i, j, k) + d_transpose(s, y[3], 1, 1, i, j, k)
             + d_transpose(s, y[4], 2, 1, i, j, k);
    out[1] = d_transpose(s, y[1], 1, 0, i, j, k) + d_transpose(s, y[3], 0, 1, i, j, k)
             + d_transpose(s, y[5], 2, 1, i, j, k);
    out[2] = d_transpose(s, y[2], 2, 0, i, j, k) + d_transpose(s, y[4], 0, 1, i, j, k)
             + d_transpose(s, y[5], 1, 1, i, j, k);
}

/* Transpose of div_tau: 3 velocity-like components y -> 6 stress-like. */
static void div_tau_T(const orc_sim *s, double *const y[3], long i, long j, long k, double out[6]) {
    out[0] = d_transpose(s, y[0], 0, 1, i, j, k);
    out[1] = d_transpose(s, y[1], 1, 1, i, j, k);
    out[2] = d_transpose(s, y[2], 2, 1, i, j, k);
    out[3] = d_transpose(s, y[0], 1, 0, i, j, k) + d_transpose(s, y[1], 0, 0, i, j, k);
    out[4] = d_transpose(s, y[0], 2, 0, i, j, k) + d_transpose(s, y[2], 0, 0, i, j, k);
    out[5] = d_transpose(s, y[1], 2, 0, i, j, k) + d_transpose(s, y[2], 1, 0, i, j, k);
}

/* mu at the cell from the stored lambda and lambda + 2 mu. */
static double cell_mu(const orc_sim *s, long c) { return 0.5 * (s->lp2m[c] - s->lam[c]); }

/* d(shear mean)/d(mu of cell m) for the 4 cells c4 of one xz or yz shear
 * point on plane k: 1/4 (arithmetic, R4), or mean^2 / (4 mu_m^2) on the
 * surface plane (harmonic, R16). */
static double shear_weight(const orc_sim *s, long k, const long c4[4], int m, double mean) {
    if (s->fs >= 1 && k == s->fs - 1) {
        double mu = cell_mu(s, c4[m]);
        return mean * mean / (4.0 * mu * mu);
    }
    return 0.25;
}

/* Reading R16: the medium above the surface is eps times the surface cell
 * of its column, so a derivative with respect to the effective medium there
 * belongs to that cell (times eps); the input values above it are unused. */
static void fold_vacuum(const orc_sim *s, double *g) {
    if (s->fs < 1) return;
    for (long j = 0; j < s->ny; ++j)
        for (long i = 0; i < s->nx; ++i) {
            double sum = 0.0;
            for (long k = 0; k < s->fs; ++k) {
                sum += g[IDX(s, i, j, k)];
                g[IDX(s, i, j, k)] = 0.0;
            }
            g[IDX(s, i, j, s->fs)] += s->fs_eps * sum;
        }
}

int orc_gradient(orc_sim *s, int nt, double dt, int src_kind, const double *pos,
                 const double *comp, const double *wavelet, int nrec, const double *rpos,
                 const double *sadj, int ckpt_every, double *g_lam, double *g_mu, double *g_rho) {
    if (s->boundary == BND_CPML) return -3;
    const long N = s->n, nx = s->nx, ny = s->ny, nz = s->nz;
    const int K = ckpt_every > 0 ? ckpt_every : nt;
    const int nck = (nt + K - 1) / K;
    double *ck = (double *)calloc((size_t)nck * NFIELD * N, sizeof(double));
    double *hist = (double *)calloc((size_t)K * (NFIELD + 3) * N, sizeof(double));
    double *av[3], *as[6], *w[6], *tmp[3], *acc[8];
    for (int q = 0; q < 3; ++q) { av[q] = zalloc(N); tmp[q] = zalloc(N); }
    for (int q = 0; q < 6; ++q) { as[q] = zalloc(N); w[q] = zalloc(N); }
    for (int q = 0; q < 8; ++q) acc[q] = zalloc(N);
    const double vol = s->h[0] * s->h[1] * s->h[2];
    int rc = 0;
    for (int q = 0; q < NFIELD; ++q) memset(s->f[q], 0, sizeof(double) * N);
    /* forward pass, checkpoint before steps 0, K, 2K, ... */
    for (int n = 0; n < nt; ++n) {
        if (n % K == 0) orc_get_state(s, ck + (size_t)(n / K) * NFIELD * N);
        if (orc_step_velocity(s, dt, src_kind, pos, comp, wavelet[n]) != 0 ||
            orc_step_stress(s, dt, src_kind, pos, comp, wavelet[n]) != 0) { rc = -1; goto done; }
    }
    for (int c = nck - 1; c >= 0; --c) {
        const int n0 = c * K, n1 = (n0 + K < nt) ? n0 + K : nt;
        orc_set_state(s, ck + (size_t)c * NFIELD * N);
        /* recompute the segment: state before step n, then v^{n+1/2} */
        for (int n = n0; n < n1; ++n) {
            double *hn = hist + (size_t)(n - n0) * (NFIELD + 3) * N;
            orc_get_state(s, hn);
            orc_step_velocity(s, dt, src_kind, pos, comp, wavelet[n]);
            for (int q = 0; q < 3; ++q) memcpy(hn + (NFIELD + q) * N, s->f[q], sizeof(double) * N);
            orc_step_stress(s, dt, src_kind, pos, comp, wavelet[n]);
        }
        for (int n = n1 - 1; n >= n0; --n) {
            double *hn = hist + (size_t)(n - n0) * (NFIELD + 3) * N;
            double *sig[6], *vh[3];
            for (int q = 0; q < 6; ++q) sig[q] = hn + (3 + q) * N;     /* sigma^n  */
            for (int q = 0; q < 3; ++q) vh[q] = hn + (NFIELD + q) * N; /* v^{n+1/2} */
            /* reverse of T */
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        long cc = IDX(s, i, j, k);
                        double G = s->g[0][i] * s->g[1][j] * s->g[2][k];
                        for (int q = 0; q < 6; ++q) w[q][cc] = G * as[q][cc];
                    }
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        long cc = IDX(s, i, j, k);
                        double e[6];
                        grad_q(s, vh, i, j, k, e);
                        double l = s->lam[cc], mu = 0.5 * (s->lp2m[cc] - l);
                        double tr = e[0] + e[1] + e[2], wtr = w[0][cc] + w[1][cc] + w[2][cc];
                        acc[0][cc] += dt * tr * wtr;                                   /* lambda   */
                        acc[1][cc] += dt * 2.0 * (e[0] * w[0][cc] + e[1] * w[1][cc] + e[2] * w[2][cc]);
                        acc[2][cc] += dt * e[3] * w[3][cc];                            /* mu_xy    */
                        acc[3][cc] += dt * e[4] * w[4][cc];                            /* mu_xz    */
                        acc[4][cc] += dt * e[5] * w[5][cc];                            /* mu_yz    */
                        (void)mu;
                    }
            {   /* tau = C w, kept in `as` (its old value is no longer needed) */
                for (long cc = 0; cc < N; ++cc) {
                    double l = s->lam[cc], l2m = s->lp2m[cc];
                    double a = w[0][cc], b = w[1][cc], d = w[2][cc];
                    as[0][cc] = l2m * a + l * (b + d);
                    as[1][cc] = l2m * b + l * (a + d);
                    as[2][cc] = l2m * d + l * (a + b);
                    as[3][cc] = s->mxy[cc] * w[3][cc];
                    as[4][cc] = s->mxz[cc] * w[4][cc];
                    as[5][cc] = s->myz[cc] * w[5][cc];
                }
                #pragma omp parallel for
                for (long k = 0; k < nz; ++k)
                    for (long j = 0; j < ny; ++j)
                        for (long i = 0; i < nx; ++i) {
                            long cc = IDX(s, i, j, k);
                            double dv[3];
                            grad_q_T(s, as, i, j, k, dv);
                            for (int q = 0; q < 3; ++q) tmp[q][cc] = dv[q];
                        }
                for (int q = 0; q < 3; ++q)
                    for (long cc = 0; cc < N; ++cc) av[q][cc] += dt * tmp[q][cc];
            }
            /* receivers: a_v += S^T sadj_n */
            for (int r = 0; r < nrec; ++r)
                for (int q = 0; q < 3; ++q) {
                    long idx[8]; double wt[8];
                    trilinear(s, q, rpos + 3 * r, idx, wt);
                    double a = sadj[((long)q * nrec + r) * nt + n];
                    for (int m = 0; m < 8; ++m)
                        if (idx[m] >= 0) av[q][idx[m]] += wt[m] * a;
                }
            for (int q = 0; q < 6; ++q) memcpy(as[q], w[q], sizeof(double) * N);
            /* reverse of V */
            const double *b[3] = {s->bx, s->by, s->bz};
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        long cc = IDX(s, i, j, k);
                        double G = s->g[0][i] * s->g[1][j] * s->g[2][k];
                        double dsig[3];
                        div_tau(s, sig, i, j, k, dsig);
                        for (int q = 0; q < 3; ++q) {
                            double u = G * av[q][cc];
                            av[q][cc] = u;
                            acc[5 + q][cc] += dt * dsig[q] * u;
                            tmp[q][cc] = b[q][cc] * u;                 /* q = B u */
                        }
                    }
            if (src_kind == 1) {   /* force term f_n / b at the taps */
                for (int q = 0; q < 3; ++q) {
                    long idx[8]; double wt[8];
                    trilinear(s, q, pos, idx, wt);
                    for (int m = 0; m < 8; ++m)
                        if (idx[m] >= 0)
                            acc[5 + q][idx[m]] += wt[m] * dt * comp[q] * wavelet[n] / vol * av[q][idx[m]];
                }
            }
            #pragma omp parallel for
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        long cc = IDX(s, i, j, k);
                        double e[6];
                        div_tau_T(s, tmp, i, j, k, e);
                        for (int q = 0; q < 6; ++q) w[q][cc] = e[q];
                    }
            for (int q = 0; q < 6; ++q)
                for (long cc = 0; cc < N; ++cc) as[q][cc] += dt * w[q][cc];
        }
    }
    /* medium chain rule: lambda direct; mu normal + 1/4 of each shear mean;
     * rho through b = 1 / (mean of 2 densities). */
    for (long cc = 0; cc < N; ++cc) { g_lam[cc] = acc[0][cc]; g_mu[cc] = acc[1][cc]; g_rho[cc] = 0.0; }
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long cc = IDX(s, i, j, k);
                long ip = clampi(i + 1, nx), jp = clampi(j + 1, ny), kp = clampi(k + 1, nz);
                long xy[4] = {cc, IDX(s, ip, j, k), IDX(s, i, jp, k), IDX(s, ip, jp, k)};
                long xz[4] = {cc, IDX(s, ip, j, k), IDX(s, i, j, kp), IDX(s, ip, j, kp)};
                long yz[4] = {cc, IDX(s, i, jp, k), IDX(s, i, j, kp), IDX(s, i, jp, kp)};
                for (int m = 0; m < 4; ++m) {
                    g_mu[xy[m]] += 0.25 * acc[2][cc];
                    g_mu[xz[m]] += shear_weight(s, k, xz, m, s->mxz[cc]) * acc[3][cc];
                    g_mu[yz[m]] += shear_weight(s, k, yz, m, s->myz[cc]) * acc[4][cc];
                }
                double bx = s->bx[cc], by = s->by[cc], bz = s->bz[cc];
                g_rho[cc] += -0.5 * bx * bx * acc[5][cc] - 0.5 * by * by * acc[6][cc] - 0.5 * bz * bz * acc[7][cc];
                g_rho[IDX(s, ip, j, k)] += -0.5 * bx * bx * acc[5][cc];
                g_rho[IDX(s, i, jp, k)] += -0.5 * by * by * acc[6][cc];
                g_rho[IDX(s, i, j, kp)] += -0.5 * bz * bz * acc[7][cc];
            }
    fold_vacuum(s, g_lam);
    fold_vacuum(s, g_mu);
    fold_vacuum(s, g_rho);
done:
    free(ck); free(hist);
    for (int q = 0; q < 3; ++q) { free(av[q]); free(tmp[q]); }
    for (int q = 0; q < 6; ++q) { free(as[q]); free(w[q]); }
    for (int q = 0; q < 8; ++q) free(acc[q]);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Tangent-linear model (forward-mode derivative of the discrete loop), for
 * the dot-product test of the adjoint: for a model perturbation dm =
 * (dlam, dmu, drho) it returns dseis = J dm exactly (to rounding), so that
 * <J dm, A> = <dm, J^T A> pins orc_gradient.  Each step differentiates the
 * operations of the forward step in order:
 *   v' = G (v + dt B Dsig(sigma) + f_n)
 *     -> dv' = G (dv + dt B Dsig(dsigma) + dt dB Dsig(sigma) + df_n),
 *        dB = -B^2 drho_mean at the v points, df_n the force term with dB;
 *   sigma' = G (sigma + dt C Dv(v') - m_n)
 *     -> dsigma' = G (dsigma + dt C Dv(dv') + dt dC Dv(v')),
 *        dC from dlam, dmu and the 4-cell means of dmu;
 *   seis_n = S v' -> dseis_n = S dv'.
 * Boundaries NONE and SPONGE (C-PML returns -3).
 * ------------------------------------------------------------------------- */

/* dv += dt dB Dsig(sigma) with the base state's stresses. */
static void velocity_tangent_extra(const orc_sim *base, orc_sim *t, double dt, const double *dbx,
                                   const double *dby, const double *dbz) {
    double *const *f = base->f;
    long nx = base->nx, ny = base->ny, nz = base->nz;
    #pragma omp parallel for
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(base, i, j, k);
                double sx = d_plus(base, f[SXX], 0, i, j, k) + d_minus(base, f[SXY], 1, i, j, k)
                            + d_minus(base, f[SXZ], 2, i, j, k);
                double sy = d_minus(base, f[SXY], 0, i, j, k) + d_plus(base, f[SYY], 1, i, j, k)
                            + d_minus(base, f[SYZ], 2, i, j, k);
                double sz = d_minus(base, f[SXZ], 0, i, j, k) + d_minus(base, f[SYZ], 1, i, j, k)
                            + d_plus(base, f[SZZ], 2, i, j, k);
                t->f[VX][c] += dt * dbx[c] * sx;
                t->f[VY][c] += dt * dby[c] * sy;
                t->f[VZ][c] += dt * dbz[c] * sz;
            }
}

/* dsigma += dt dC Dv(v') with the base state's velocities. */
static void stress_tangent_extra(const orc_sim *base, orc_sim *t, double dt, const double *dlam,
                                 const double *dl2m, const double *dmxy, const double *dmxz,
                                 const double *dmyz) {
    double *const *f = base->f;
    long nx = base->nx, ny = base->ny, nz = base->nz;
    #pragma omp parallel for
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(base, i, j, k);
                double exx = d_minus(base, f[VX], 0, i, j, k);
                double eyy = d_minus(base, f[VY], 1, i, j, k);
                double ezz = d_minus(base, f[VZ], 2, i, j, k);
                t->f[SXX][c] += dt * (dl2m[c] * exx + dlam[c] * (eyy + ezz));
                t->f[SYY][c] += dt * (dl2m[c] * eyy + dlam[c] * (exx + ezz));
                t->f[SZZ][c] += dt * (dl2m[c] * ezz + dlam[c] * (exx + eyy));
                t->f[SXY][c] += dt * dmxy[c] * (d_plus(base, f[VX], 1, i, j, k) + d_plus(base, f[VY], 0, i, j, k));
                t->f[SXZ][c] += dt * dmxz[c] * (d_plus(base, f[VX], 2, i, j, k) + d_plus(base, f[VZ], 0, i, j, k));
                t->f[SYZ][c] += dt * dmyz[c] * (d_plus(base, f[VY], 2, i, j, k) + d_plus(base, f[VZ], 1, i, j, k));
            }
}

/* dseis [3][nrec][nt] of the model perturbation (dlam, dmu, drho), from rest,
 * for the forward loop of orc_forward with the medium already set on s. */
int orc_tangent(orc_sim *s, int nt, double dt, int src_kind, const double *pos,
                const double *comp, const double *wavelet, int nrec, const double *rpos,
                const double *dlam_in, const double *dmu_in, const double *drho_in,
                double *dseis) {
    if (s->boundary == BND_CPML) return -3;
    long nx = s->nx, ny = s->ny, nz = s->nz, n = s->n;
    orc_sim *t = orc_create(nx, ny, nz, s->h[0], s->h[1], s->h[2]);
    t->fs = s->fs;
    t->fs_eps = s->fs_eps;
    /* perturbation of the effective medium: above a free surface, eps times
     * the perturbation of the column's surface cell (reading R16) */
    double *dlam = zalloc(n), *dmu = zalloc(n), *drho = zalloc(n);
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                long b = (s->fs >= 0 && k < s->fs) ? IDX(s, i, j, s->fs) : c;
                double e = b == c ? 1.0 : s->fs_eps;
                dlam[c] = e * dlam_in[b];
                dmu[c] = e * dmu_in[b];
                drho[c] = e * drho_in[b];
            }
    /* the tangent propagates with the base medium and boundary */
    memcpy(t->bx, s->bx, sizeof(double) * n); memcpy(t->by, s->by, sizeof(double) * n);
    memcpy(t->bz, s->bz, sizeof(double) * n); memcpy(t->lam, s->lam, sizeof(double) * n);
    memcpy(t->lp2m, s->lp2m, sizeof(double) * n); memcpy(t->mxy, s->mxy, sizeof(double) * n);
    memcpy(t->mxz, s->mxz, sizeof(double) * n); memcpy(t->myz, s->myz, sizeof(double) * n);
    t->boundary = s->boundary; t->width = s->width;
    for (int a = 0; a < 3; ++a) {
        long na = a == 0 ? nx : a == 1 ? ny : nz;
        memcpy(t->g[a], s->g[a], sizeof(double) * na);
    }
    /* medium perturbations at the staggered points (the means of reading R4) */
    double *dbx = zalloc(n), *dby = zalloc(n), *dbz = zalloc(n), *dl2m = zalloc(n);
    double *dmxy = zalloc(n), *dmxz = zalloc(n), *dmyz = zalloc(n);
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = IDX(s, i, j, k);
                long ip = clampi(i + 1, nx), jp = clampi(j + 1, ny), kp = clampi(k + 1, nz);
                dbx[c] = -s->bx[c] * s->bx[c] * 0.5 * (drho[c] + drho[IDX(s, ip, j, k)]);
                dby[c] = -s->by[c] * s->by[c] * 0.5 * (drho[c] + drho[IDX(s, i, jp, k)]);
                dbz[c] = -s->bz[c] * s->bz[c] * 0.5 * (drho[c] + drho[IDX(s, i, j, kp)]);
                dl2m[c] = dlam[c] + 2.0 * dmu[c];
                dmxy[c] = 0.25 * (dmu[c] + dmu[IDX(s, ip, j, k)] + dmu[IDX(s, i, jp, k)] + dmu[IDX(s, ip, jp, k)]);
                long xz[4] = {c, IDX(s, ip, j, k), IDX(s, i, j, kp), IDX(s, ip, j, kp)};
                long yz[4] = {c, IDX(s, i, jp, k), IDX(s, i, j, kp), IDX(s, i, jp, kp)};
                dmxz[c] = dmyz[c] = 0.0;
                for (int m = 0; m < 4; ++m) {
                    dmxz[c] += shear_weight(s, k, xz, m, s->mxz[c]) * dmu[xz[m]];
                    dmyz[c] += shear_weight(s, k, yz, m, s->myz[c]) * dmu[yz[m]];
                }
            }
    for (int q = 0; q < NFIELD; ++q) memset(s->f[q], 0, sizeof(double) * n);
    double *tmp = (double *)malloc(sizeof(double) * 3 * (nrec > 0 ? nrec : 1));
    double vol = s->h[0] * s->h[1] * s->h[2];
    const double *db[3] = {dbx, dby, dbz};
    int rc = 0;
    for (int it = 0; it < nt && rc == 0; ++it) {
        /* velocity: base terms of the tangent first (they use sigma^n), then the base step */
        velocity_update(t, dt);
        velocity_tangent_extra(s, t, dt, dbx, dby, dbz);
        if (src_kind == 1)
            for (int q = 0; q < 3; ++q) {
                long idx[8]; double w[8];
                if (!trilinear(s, q, pos, idx, w)) { rc = -1; break; }
                for (int m = 0; m < 8; ++m)
                    if (idx[m] >= 0) t->f[q][idx[m]] += w[m] * dt * db[q][idx[m]] * comp[q] * wavelet[it] / vol;
            }
        apply_sponge(t, VX, VZ + 1);
        if (rc == 0 && orc_step_velocity(s, dt, src_kind, pos, comp, wavelet[it]) != 0) rc = -1;
        if (rc == 0 && nrec > 0) {
            if (orc_sample(t, nrec, rpos, tmp) != 0) { rc = -2; break; }
            for (int q = 0; q < 3; ++q)
                for (int r = 0; r < nrec; ++r)
                    dseis[((long)q * nrec + r) * nt + it] = tmp[q * nrec + r];
        }
        /* stress: the tangent uses v' of the base (already stepped) */
        if (rc == 0) {
            stress_update(t, dt);
            stress_tangent_extra(s, t, dt, dlam, dl2m, dmxy, dmxz, dmyz);
            apply_sponge(t, SXX, SYZ + 1);
            if (orc_step_stress(s, dt, src_kind, pos, comp, wavelet[it]) != 0) rc = -1;
        }
    }
    free(tmp);
    free(dbx); free(dby); free(dbz); free(dl2m); free(dmxy); free(dmxz); free(dmyz);
    free(dlam); free(dmu); free(drho);
    orc_destroy(t);
    return rc;
}
