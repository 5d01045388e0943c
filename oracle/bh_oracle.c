/*
 * FP64 CPU oracle for the borehole acoustic FWI hot path
 * (Tang, Cheng, Li, Fang: "Borehole acoustic full-waveform inversion").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The CUDA library never links,
 * includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes, step by step, in double precision:
 *   - the axisymmetric monopole velocity-stress system of Eq. 2 on a
 *     staggered (r,z) grid, 4th order in space and 2nd order in time
 *     (leapfrog), with the axis symmetry condition at r = 0, a C-PML on the
 *     outer radial edge and on the top and bottom edges, a volume source in
 *     the three normal stresses, and pressure recording as the mean normal
 *     stress at the receivers (Method section, Eq. 2: the recorded data are
 *     normal stresses);
 *   - the adjoint of that discrete map (the discrete form of Eq. 6), driven
 *     by the data residual of Eq. 5.  Every loop of the forward step is
 *     transposed literally: each gather "y += w * x[k]" of the forward
 *     becomes the scatter "xbar[k] += w * ybar" here, through the same
 *     stencil tap lists, so the transpose cannot drift from the forward;
 *   - the zero-lag cross-correlations of Eq. 7 and Eq. 8 (plus the density
 *     term through the buoyancy averages) and the diagonal pseudo-Hessian
 *     used by the preconditioner;
 *   - the chain rule from node accumulators to per-cell gradients.
 *
 * Discretisation (the paper cites a finite-difference scheme but does not
 * print it; these are the readings this build fixes):
 *   cell (i,j)  at r=(i+1/2)dr, z=j dz      : trr, ttt, tzz, lambda, mu, rho
 *   v_r  (i,j)  at r=i dr,      z=j dz      : v_r(0,j) = 0 on the axis
 *   v_z  (i,j)  at r=(i+1/2)dr, z=(j+1/2)dz
 *   trz  (i,j)  at r=i dr,      z=(j+1/2)dz : trz(0,j) = 0 on the axis
 *   D f = [c1 (f(+1/2) - f(-1/2)) + c2 (f(+3/2) - f(-3/2))] / h,
 *         c1 = 9/8, c2 = -1/24.
 *   1/r terms: two-point average to the target node over the target's r.
 *   Axis ghosts: half-r fields mirror evenly (f[-1-k] = f[k]); integer-r
 *   fields mirror oddly (f[-k] = -f[k], f[0] = 0).  Beyond r >= nr and
 *   outside 0 <= z < nz every ghost is zero.
 *   C-PML: recursive convolution with kappa = 1,
 *     psi <- b psi + a D u,  the step uses D u + psi,
 *     d = d0 x^2, d0 = -3 Vpmax ln(R) / (2 L), alpha = pi f0 (1 - x),
 *     b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha).
 *
 * The gradient is reported for the cells outside the absorbing layers only
 * (the model inside the C-PML is a fixed extension, not an unknown).  Every
 * node that touches such a cell has a = 0, so its memory variable is zero at
 * all times and the correlation needs no stored psi history.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nr, nz, nt, npml_r, npml_z;
    double dr, dz, dt, f0, pml_R, vpmax;
} orc_grid;

#define C1 (9.0 / 8.0)
#define C2 (-1.0 / 24.0)

enum { LOC_INT = 0, LOC_HALF = 1 };

/* A stencil after the boundary rules: up to 4 (flat index, weight) terms. */
typedef struct {
    int n;
    long idx[4];
    double w[4];
} taps_t;

/* Radial index k of a field living at integer (LOC_INT) or half (LOC_HALF)
 * radial positions, mapped through the axis mirror and the outer zero edge.
 * Returns 0 when the value there is identically zero. */
static int map_r(int loc, int k, int nr, int *kk, double *sgn)
{
    double s = 1.0;
    if (loc == LOC_HALF) {
        if (k < 0) k = -1 - k;              /* even mirror about r = 0 */
    } else {
        if (k == 0) return 0;               /* v_r, trz vanish on the axis */
        if (k < 0) { k = -k; s = -1.0; }    /* odd mirror about r = 0 */
    }
    if (k >= nr) return 0;
    *kk = k;
    *sgn = s;
    return 1;
}

/* 4th-order radial difference at target radial index i (row of the target
 * node), reading a field located at `src`.  The target sits at the other
 * kind of position.  Column j is fixed. */
static void taps_dr(int src, int i, int j, int nr, int nz, double dr, taps_t *t)
{
    static const int off_from_half[4] = {0, -1, 1, -2}; /* target at i      */
    static const int off_from_int[4] = {1, 0, 2, -1};   /* target at i+1/2  */
    const double w[4] = {C1, -C1, C2, -C2};
    const int *off = (src == LOC_HALF) ? off_from_half : off_from_int;
    t->n = 0;
    for (int q = 0; q < 4; ++q) {
        int kk;
        double s;
        if (map_r(src, i + off[q], nr, &kk, &s)) {
            t->idx[t->n] = (long)kk * nz + j;
            t->w[t->n] = s * w[q] / dr;
            t->n++;
        }
    }
}

/* 4th-order axial difference at target column j; `src` is the axial
 * location of the field read (LOC_INT: z = j dz, LOC_HALF: z = (j+1/2) dz). */
static void taps_dz(int src, int i, int j, int nz, double dz, taps_t *t)
{
    static const int off_from_half[4] = {0, -1, 1, -2};
    static const int off_from_int[4] = {1, 0, 2, -1};
    const double w[4] = {C1, -C1, C2, -C2};
    const int *off = (src == LOC_HALF) ? off_from_half : off_from_int;
    t->n = 0;
    for (int q = 0; q < 4; ++q) {
        int k = j + off[q];
        if (k >= 0 && k < nz) {
            t->idx[t->n] = (long)i * nz + k;
            t->w[t->n] = w[q] / dz;
            t->n++;
        }
    }
}

/* Two-point radial average to target row i, divided by the target radius. */
static void taps_avg_over_r(int src, int i, int j, int nr, int nz, double r_target, taps_t *t)
{
    static const int off_from_half[2] = {-1, 0}; /* target at integer r   */
    static const int off_from_int[2] = {0, 1};   /* target at half r      */
    const int *off = (src == LOC_HALF) ? off_from_half : off_from_int;
    t->n = 0;
    for (int q = 0; q < 2; ++q) {
        int kk;
        double s;
        if (map_r(src, i + off[q], nr, &kk, &s)) {
            t->idx[t->n] = (long)kk * nz + j;
            t->w[t->n] = s * 0.5 / r_target;
            t->n++;
        }
    }
}

static double gather(const double *f, const taps_t *t)
{
    double acc = 0.0;
    for (int q = 0; q < t->n; ++q) acc += t->w[q] * f[t->idx[q]];
    return acc;
}

static void scatter(double *f, const taps_t *t, double x)
{
    for (int q = 0; q < t->n; ++q) f[t->idx[q]] += t->w[q] * x;
}

/* ------------------------------------------------------------------ */
/* Model and coefficients                                              */

typedef struct {
    orc_grid g;
    long ncell;
    double *lam, *mu, *rho;      /* per cell (Eq. 3, Eq. 4)                */
    double *bvr, *bvz, *muh;     /* buoyancy at v nodes, harmonic mu at trz */
    double *r_int, *r_half;      /* [nr]                                    */
    double *ar_int, *br_int, *ar_half, *br_half;  /* radial C-PML, [nr]    */
    double *az_int, *bz_int, *az_half, *bz_half;  /* axial C-PML, [nz]     */
} model_t;

static void pml_ab(double x, double d0, double alpha_max, double dt, double *a, double *b)
{
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    double d = d0 * x * x;
    double alpha = alpha_max * (1.0 - x);
    *b = exp(-(d + alpha) * dt);
    *a = (d > 0.0) ? d * (*b - 1.0) / (d + alpha) : 0.0;
}

static int model_init(model_t *m, const orc_grid *g, const double *vp, const double *vs,
                      const double *rho)
{
    memset(m, 0, sizeof(*m));
    m->g = *g;
    int nr = g->nr, nz = g->nz;
    long nc = (long)nr * nz;
    m->ncell = nc;
    double *blk = (double *)calloc((size_t)(6 * nc + 6 * nr + 4 * nz), sizeof(double));
    if (!blk) return -1;
    m->lam = blk;
    m->mu = blk + nc;
    m->rho = blk + 2 * nc;
    m->bvr = blk + 3 * nc;
    m->bvz = blk + 4 * nc;
    m->muh = blk + 5 * nc;
    double *p = blk + 6 * nc;
    m->r_int = p; p += nr;
    m->r_half = p; p += nr;
    m->ar_int = p; p += nr;
    m->br_int = p; p += nr;
    m->ar_half = p; p += nr;
    m->br_half = p; p += nr;
    m->az_int = p; p += nz;
    m->bz_int = p; p += nz;
    m->az_half = p; p += nz;
    m->bz_half = p; p += nz;

    for (long c = 0; c < nc; ++c) {
        /* Eq. 3 and Eq. 4 */
        m->rho[c] = rho[c];
        m->mu[c] = rho[c] * vs[c] * vs[c];
        m->lam[c] = rho[c] * vp[c] * vp[c] - 2.0 * rho[c] * vs[c] * vs[c];
    }
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            int jp = (j + 1 < nz) ? j + 1 : nz - 1; /* axial edge: the single cell */
            /* buoyancy at v_r (i,j): mean of 1/rho over cells i-1, i */
            if (i >= 1) m->bvr[c] = 0.5 * (1.0 / m->rho[c - nz] + 1.0 / m->rho[c]);
            /* buoyancy at v_z (i,j): mean of 1/rho over cells j, j+1 */
            m->bvz[c] = 0.5 * (1.0 / m->rho[c] + 1.0 / m->rho[(long)i * nz + jp]);
            /* harmonic mean of mu over the 4 cells around trz (i,j) */
            if (i >= 1) {
                const double q[4] = {m->mu[(long)(i - 1) * nz + j], m->mu[(long)i * nz + j],
                                     m->mu[(long)(i - 1) * nz + jp], m->mu[(long)i * nz + jp]};
                int zero = 0;
                double s = 0.0;
                for (int k = 0; k < 4; ++k) {
                    if (q[k] <= 0.0) zero = 1;
                    else s += 1.0 / q[k];
                }
                m->muh[c] = zero ? 0.0 : 4.0 / s;
            }
        }

    for (int i = 0; i < nr; ++i) {
        m->r_int[i] = i * g->dr;
        m->r_half[i] = (i + 0.5) * g->dr;
    }
    const double alpha_max = M_PI * g->f0;
    const double R = g->pml_R > 0.0 ? g->pml_R : 1e-3;
    /* radial layer: r from (nr - npml_r) dr to nr dr */
    double Lr = g->npml_r * g->dr;
    double d0r = (g->npml_r > 0) ? -3.0 * g->vpmax * log(R) / (2.0 * Lr) : 0.0;
    for (int i = 0; i < nr; ++i) {
        double xi = (g->npml_r > 0) ? (m->r_int[i] - (nr - g->npml_r) * g->dr) / Lr : 0.0;
        double xh = (g->npml_r > 0) ? (m->r_half[i] - (nr - g->npml_r) * g->dr) / Lr : 0.0;
        pml_ab(xi, d0r, alpha_max, g->dt, &m->ar_int[i], &m->br_int[i]);
        pml_ab(xh, d0r, alpha_max, g->dt, &m->ar_half[i], &m->br_half[i]);
    }
    /* axial layers: the top one ends at z = (npml_z - 1/2) dz, the bottom one
     * starts at z = (nz - npml_z - 1/2) dz; cells sit at z = j dz. */
    double Lz = g->npml_z * g->dz;
    double d0z = (g->npml_z > 0) ? -3.0 * g->vpmax * log(R) / (2.0 * Lz) : 0.0;
    for (int j = 0; j < nz; ++j) {
        for (int h = 0; h < 2; ++h) {
            double z = (j + 0.5 * h) * g->dz;
            double x = 0.0;
            if (g->npml_z > 0) {
                double xt = ((g->npml_z - 0.5) * g->dz - z) / Lz;
                double xb = (z - (nz - g->npml_z - 0.5) * g->dz) / Lz;
                x = xt > xb ? xt : xb;
            }
            if (h == 0) pml_ab(x, d0z, alpha_max, g->dt, &m->az_int[j], &m->bz_int[j]);
            else pml_ab(x, d0z, alpha_max, g->dt, &m->az_half[j], &m->bz_half[j]);
        }
    }
    return 0;
}

static void model_free(model_t *m) { free(m->lam); }

/* ------------------------------------------------------------------ */
/* Wavefield state                                                     */

enum { F_VR = 0, F_VZ, F_TRR, F_TTT, F_TZZ, F_TRZ, NFIELD };
/* C-PML memory variables, by the derivative they stretch:
 * 0 d/dr trr @v_r, 1 d/dz trz @v_r, 2 d/dr trz @v_z, 3 d/dz tzz @v_z,
 * 4 d/dr v_r @cell, 5 d/dz v_z @cell, 6 d/dz v_r @trz, 7 d/dr v_z @trz */
#define NPSI 8

typedef struct {
    double *f[NFIELD];
    double *psi[NPSI];
    double *blk;
} state_t;

static int state_alloc(state_t *s, long nc)
{
    s->blk = (double *)calloc((size_t)(NFIELD + NPSI) * nc, sizeof(double));
    if (!s->blk) return -1;
    for (int k = 0; k < NFIELD; ++k) s->f[k] = s->blk + k * nc;
    for (int k = 0; k < NPSI; ++k) s->psi[k] = s->blk + (NFIELD + k) * nc;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Forward: Eq. 2 lines 1-2 (velocities), then lines 3-6 (stresses).   */

static void velocity_step(const model_t *m, state_t *s)
{
    const orc_grid *g = &m->g;
    const int nr = g->nr, nz = g->nz;
    double *vr = s->f[F_VR], *vz = s->f[F_VZ];
    const double *trr = s->f[F_TRR], *ttt = s->f[F_TTT], *tzz = s->f[F_TZZ], *trz = s->f[F_TRZ];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; ++i) {
        taps_t t;
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            if (i >= 1) {
                /* v_r: d trr/dr + d trz/dz + (trr - ttt)/r */
                taps_dr(LOC_HALF, i, j, nr, nz, g->dr, &t);
                double d_trr_dr = gather(trr, &t);
                taps_dz(LOC_HALF, i, j, nz, g->dz, &t);
                double d_trz_dz = gather(trz, &t);
                taps_avg_over_r(LOC_HALF, i, j, nr, nz, m->r_int[i], &t);
                double hoop = gather(trr, &t) - gather(ttt, &t);
                s->psi[0][c] = m->br_int[i] * s->psi[0][c] + m->ar_int[i] * d_trr_dr;
                s->psi[1][c] = m->bz_int[j] * s->psi[1][c] + m->az_int[j] * d_trz_dz;
                vr[c] += g->dt * m->bvr[c] *
                         (d_trr_dr + s->psi[0][c] + d_trz_dz + s->psi[1][c] + hoop);
            }
            /* v_z: d trz/dr + d tzz/dz + trz/r */
            taps_dr(LOC_INT, i, j, nr, nz, g->dr, &t);
            double d_trz_dr = gather(trz, &t);
            taps_dz(LOC_INT, i, j, nz, g->dz, &t);
            double d_tzz_dz = gather(tzz, &t);
            taps_avg_over_r(LOC_INT, i, j, nr, nz, m->r_half[i], &t);
            double hoop = gather(trz, &t);
            s->psi[2][c] = m->br_half[i] * s->psi[2][c] + m->ar_half[i] * d_trz_dr;
            s->psi[3][c] = m->bz_half[j] * s->psi[3][c] + m->az_half[j] * d_tzz_dz;
            vz[c] += g->dt * m->bvz[c] * (d_trz_dr + s->psi[2][c] + d_tzz_dz + s->psi[3][c] + hoop);
        }
    }
}

static void stress_step(const model_t *m, state_t *s)
{
    const orc_grid *g = &m->g;
    const int nr = g->nr, nz = g->nz;
    const double *vr = s->f[F_VR], *vz = s->f[F_VZ];
    double *trr = s->f[F_TRR], *ttt = s->f[F_TTT], *tzz = s->f[F_TZZ], *trz = s->f[F_TRZ];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; ++i) {
        taps_t t;
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            /* cell: normal strains */
            taps_dr(LOC_INT, i, j, nr, nz, g->dr, &t);
            double d_vr_dr = gather(vr, &t);
            taps_avg_over_r(LOC_INT, i, j, nr, nz, m->r_half[i], &t);
            double vr_over_r = gather(vr, &t);
            taps_dz(LOC_HALF, i, j, nz, g->dz, &t);
            double d_vz_dz = gather(vz, &t);
            s->psi[4][c] = m->br_half[i] * s->psi[4][c] + m->ar_half[i] * d_vr_dr;
            s->psi[5][c] = m->bz_int[j] * s->psi[5][c] + m->az_int[j] * d_vz_dz;
            double err = d_vr_dr + s->psi[4][c];
            double ett = vr_over_r;
            double ezz = d_vz_dz + s->psi[5][c];
            double lam = m->lam[c], l2m = m->lam[c] + 2.0 * m->mu[c];
            trr[c] += g->dt * (l2m * err + lam * ett + lam * ezz);
            ttt[c] += g->dt * (lam * err + l2m * ett + lam * ezz);
            tzz[c] += g->dt * (lam * err + lam * ett + l2m * ezz);
            /* trz node */
            if (i >= 1) {
                taps_dz(LOC_INT, i, j, nz, g->dz, &t);
                double d_vr_dz = gather(vr, &t);
                taps_dr(LOC_HALF, i, j, nr, nz, g->dr, &t);
                double d_vz_dr = gather(vz, &t);
                s->psi[6][c] = m->bz_half[j] * s->psi[6][c] + m->az_half[j] * d_vr_dz;
                s->psi[7][c] = m->br_int[i] * s->psi[7][c] + m->ar_int[i] * d_vz_dr;
                trz[c] += g->dt * m->muh[c] * (d_vr_dz + s->psi[6][c] + d_vz_dr + s->psi[7][c]);
            }
        }
    }
}

static double source_volume(const model_t *m, int src_ir)
{
    const orc_grid *g = &m->g;
    if (src_ir == 0) return M_PI * g->dr * g->dr * g->dz;  /* disk on the axis */
    return 2.0 * M_PI * m->r_half[src_ir] * g->dr * g->dz; /* ring */
}

/*
 * Forward modelling.
 *   wavelet [nt]      : source rate s(t_{n+1/2}) injected at step n
 *   seis    [nrec][nt]: mean normal stress at (0, rec_iz[k]) after step n
 *   vhist   [nt][2][nr*nz] or NULL: v_r, v_z at t_{n+1/2}
 *   force   [nt][6][nr*nz] or NULL: added to each field after its update
 *           (used by the adjoint dot-product test only)
 */
int orc_forward(const orc_grid *g, const double *vp, const double *vs, const double *rho,
                const double *wavelet, int src_ir, int src_iz, int nrec, const int *rec_iz,
                double *seis, double *vhist, const double *force)
{
    model_t m;
    state_t s;
    if (model_init(&m, g, vp, vs, rho)) return -1;
    long nc = m.ncell;
    if (state_alloc(&s, nc)) { model_free(&m); return -1; }
    const double vsrc = source_volume(&m, src_ir);
    const long csrc = (long)src_ir * g->nz + src_iz;
    for (int n = 0; n < g->nt; ++n) {
        velocity_step(&m, &s);
        if (force) {
            const double *fn = force + (long)n * NFIELD * nc;
            for (long c = 0; c < nc; ++c) {
                if (c >= g->nz) s.f[F_VR][c] += fn[c];   /* v_r(0,.) stays 0 */
                s.f[F_VZ][c] += fn[nc + c];
            }
        }
        if (vhist) {
            memcpy(vhist + (long)n * 2 * nc, s.f[F_VR], nc * sizeof(double));
            memcpy(vhist + (long)n * 2 * nc + nc, s.f[F_VZ], nc * sizeof(double));
        }
        stress_step(&m, &s);
        const double inj = g->dt * wavelet[n] / vsrc;
        s.f[F_TRR][csrc] += inj;
        s.f[F_TTT][csrc] += inj;
        s.f[F_TZZ][csrc] += inj;
        if (force) {
            const double *fn = force + (long)n * NFIELD * nc;
            for (long c = 0; c < nc; ++c) {
                s.f[F_TRR][c] += fn[2 * nc + c];
                s.f[F_TTT][c] += fn[3 * nc + c];
                s.f[F_TZZ][c] += fn[4 * nc + c];
                if (c >= g->nz) s.f[F_TRZ][c] += fn[5 * nc + c];  /* trz(0,.) stays 0 */
            }
        }
        for (int k = 0; k < nrec; ++k) {
            long c = rec_iz[k]; /* receivers sit in cell i = 0 on the axis */
            seis[(long)k * g->nt + n] =
                (s.f[F_TRR][c] + s.f[F_TTT][c] + s.f[F_TZZ][c]) / 3.0;
        }
    }
    free(s.blk);
    model_free(&m);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adjoint: literal transpose of the two steps above.                  */

/* transpose of velocity_step: reads Av (and the adjoint C-PML memories of
 * the velocity step), adds into Atau. */
static void velocity_step_T(const model_t *m, state_t *a)
{
    const orc_grid *g = &m->g;
    const int nr = g->nr, nz = g->nz;
    const double *avr = a->f[F_VR], *avz = a->f[F_VZ];
    double *atrr = a->f[F_TRR], *attt = a->f[F_TTT], *atzz = a->f[F_TZZ], *atrz = a->f[F_TRZ];
    taps_t t;
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            if (i >= 1) {
                double w = g->dt * m->bvr[c] * avr[c]; /* adjoint of the bracket */
                a->psi[0][c] = w + m->br_int[i] * a->psi[0][c];
                a->psi[1][c] = w + m->bz_int[j] * a->psi[1][c];
                double x0 = w + m->ar_int[i] * a->psi[0][c];
                double x1 = w + m->az_int[j] * a->psi[1][c];
                taps_dr(LOC_HALF, i, j, nr, nz, g->dr, &t);
                scatter(atrr, &t, x0);
                taps_dz(LOC_HALF, i, j, nz, g->dz, &t);
                scatter(atrz, &t, x1);
                taps_avg_over_r(LOC_HALF, i, j, nr, nz, m->r_int[i], &t);
                scatter(atrr, &t, w);
                scatter(attt, &t, -w);
            }
            double w = g->dt * m->bvz[c] * avz[c];
            a->psi[2][c] = w + m->br_half[i] * a->psi[2][c];
            a->psi[3][c] = w + m->bz_half[j] * a->psi[3][c];
            double x2 = w + m->ar_half[i] * a->psi[2][c];
            double x3 = w + m->az_half[j] * a->psi[3][c];
            taps_dr(LOC_INT, i, j, nr, nz, g->dr, &t);
            scatter(atrz, &t, x2);
            taps_dz(LOC_INT, i, j, nz, g->dz, &t);
            scatter(atzz, &t, x3);
            taps_avg_over_r(LOC_INT, i, j, nr, nz, m->r_half[i], &t);
            scatter(atrz, &t, w);
        }
}

/* transpose of stress_step: reads Atau (and the adjoint memories of the
 * stress step), adds into Av. */
static void stress_step_T(const model_t *m, state_t *a)
{
    const orc_grid *g = &m->g;
    const int nr = g->nr, nz = g->nz;
    double *avr = a->f[F_VR], *avz = a->f[F_VZ];
    const double *atrr = a->f[F_TRR], *attt = a->f[F_TTT], *atzz = a->f[F_TZZ],
                 *atrz = a->f[F_TRZ];
    taps_t t;
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            double lam = m->lam[c], l2m = m->lam[c] + 2.0 * m->mu[c];
            /* adjoints of err, ett, ezz (transpose of the stiffness matrix) */
            double y_rr = g->dt * (l2m * atrr[c] + lam * attt[c] + lam * atzz[c]);
            double y_tt = g->dt * (lam * atrr[c] + l2m * attt[c] + lam * atzz[c]);
            double y_zz = g->dt * (lam * atrr[c] + lam * attt[c] + l2m * atzz[c]);
            a->psi[4][c] = y_rr + m->br_half[i] * a->psi[4][c];
            a->psi[5][c] = y_zz + m->bz_int[j] * a->psi[5][c];
            double x4 = y_rr + m->ar_half[i] * a->psi[4][c];
            double x5 = y_zz + m->az_int[j] * a->psi[5][c];
            taps_dr(LOC_INT, i, j, nr, nz, g->dr, &t);
            scatter(avr, &t, x4);
            taps_avg_over_r(LOC_INT, i, j, nr, nz, m->r_half[i], &t);
            scatter(avr, &t, y_tt);
            taps_dz(LOC_HALF, i, j, nz, g->dz, &t);
            scatter(avz, &t, x5);
            if (i >= 1) {
                double y = g->dt * m->muh[c] * atrz[c];
                a->psi[6][c] = y + m->bz_half[j] * a->psi[6][c];
                a->psi[7][c] = y + m->br_int[i] * a->psi[7][c];
                double x6 = y + m->az_half[j] * a->psi[6][c];
                double x7 = y + m->ar_int[i] * a->psi[7][c];
                taps_dz(LOC_INT, i, j, nz, g->dz, &t);
                scatter(avr, &t, x6);
                taps_dr(LOC_HALF, i, j, nr, nz, g->dr, &t);
                scatter(avz, &t, x7);
            }
        }
}

/* Accumulator planes written by orc_adjoint. */
enum {
    G_LAM = 0, /* cell:  sum dt div(v) (Atrr + Attt + Atzz)               (Eq. 7) */
    G_MUNN,    /* cell:  sum dt 2 (err Atrr + ett Attt + ezz Atzz)       (Eq. 8) */
    G_MURZ,    /* trz:   sum dt (dv_r/dz + dv_z/dr) Atrz                  (Eq. 8) */
    G_BR,      /* v_r:   sum dt F_r Av_r, F_r the bracket of Eq. 2 line 1        */
    G_BZ,      /* v_z:   sum dt F_z Av_z                                         */
    H_LAM,     /* cell:  sum dt div(v)^2        (pseudo-Hessian, lambda)        */
    H_MUNN,    /* cell:  sum dt 4 (err^2 + ett^2 + ezz^2)                       */
    H_MURZ,    /* trz:   sum dt (dv_r/dz + dv_z/dr)^2                           */
    NACC
};

/*
 * Adjoint modelling and gradient correlation.
 *   resid  [nrec][nt]: data residual (Eq. 5), adjoint source Δp/3 into each
 *                      of the three normal stresses at the receiver cell
 *   vhist  [nt][2][nr*nz]: forward v_r, v_z at t_{n+1/2}
 *   acc    [NACC][nr*nz]: correlation accumulators (output)
 *   wavelet_bar [nt] or NULL: adjoint of the source wavelet
 *   force_bar [nt][6][nr*nz] or NULL: adjoint of the forcing of orc_forward
 */
int orc_adjoint(const orc_grid *g, const double *vp, const double *vs, const double *rho,
                const double *resid, int src_ir, int src_iz, int nrec, const int *rec_iz,
                const double *vhist, double *acc, double *wavelet_bar, double *force_bar)
{
    model_t m;
    state_t a;
    if (model_init(&m, g, vp, vs, rho)) return -1;
    const int nr = g->nr, nz = g->nz;
    long nc = m.ncell;
    if (state_alloc(&a, nc)) { model_free(&m); return -1; }
    memset(acc, 0, (size_t)NACC * nc * sizeof(double));
    const double vsrc = source_volume(&m, src_ir);
    const long csrc = (long)src_ir * nz + src_iz;
    taps_t t;
    for (int n = g->nt - 1; n >= 0; --n) {
        /* transpose of the recording: Δp/3 into each normal stress */
        for (int k = 0; k < nrec; ++k) {
            long c = rec_iz[k];
            double r3 = resid[(long)k * g->nt + n] / 3.0;
            a.f[F_TRR][c] += r3;
            a.f[F_TTT][c] += r3;
            a.f[F_TZZ][c] += r3;
        }
        if (wavelet_bar)
            wavelet_bar[n] = g->dt / vsrc *
                             (a.f[F_TRR][csrc] + a.f[F_TTT][csrc] + a.f[F_TZZ][csrc]);
        if (force_bar) {
            double *fb = force_bar + (long)n * NFIELD * nc;
            for (long c = 0; c < nc; ++c) {
                fb[2 * nc + c] = a.f[F_TRR][c];
                fb[3 * nc + c] = a.f[F_TTT][c];
                fb[4 * nc + c] = a.f[F_TZZ][c];
                fb[5 * nc + c] = (c >= nz) ? a.f[F_TRZ][c] : 0.0;
            }
        }

        /* gradient correlation of Eq. 7 / Eq. 8 at step n, using the forward
         * strains of v^{n+1/2} and Atau = dJ/dtau^{n+1} */
        const double *vr = vhist + (long)n * 2 * nc, *vz = vr + nc;
        for (int i = 0; i < nr; ++i)
            for (int j = 0; j < nz; ++j) {
                long c = (long)i * nz + j;
                taps_dr(LOC_INT, i, j, nr, nz, g->dr, &t);
                double err = gather(vr, &t);
                taps_avg_over_r(LOC_INT, i, j, nr, nz, m.r_half[i], &t);
                double ett = gather(vr, &t);
                taps_dz(LOC_HALF, i, j, nz, g->dz, &t);
                double ezz = gather(vz, &t);
                double div = err + ett + ezz;
                double sum_a = a.f[F_TRR][c] + a.f[F_TTT][c] + a.f[F_TZZ][c];
                acc[G_LAM * nc + c] += g->dt * div * sum_a;
                acc[G_MUNN * nc + c] += g->dt * 2.0 *
                    (err * a.f[F_TRR][c] + ett * a.f[F_TTT][c] + ezz * a.f[F_TZZ][c]);
                acc[H_LAM * nc + c] += g->dt * div * div;
                acc[H_MUNN * nc + c] += g->dt * 4.0 * (err * err + ett * ett + ezz * ezz);
                if (i >= 1) {
                    taps_dz(LOC_INT, i, j, nz, g->dz, &t);
                    double gam = gather(vr, &t);
                    taps_dr(LOC_HALF, i, j, nr, nz, g->dr, &t);
                    gam += gather(vz, &t);
                    acc[G_MURZ * nc + c] += g->dt * gam * a.f[F_TRZ][c];
                    acc[H_MURZ * nc + c] += g->dt * gam * gam;
                }
            }

        stress_step_T(&m, &a);   /* Av now holds dJ/dv^{n+1/2} */

        if (force_bar) {
            double *fb = force_bar + (long)n * NFIELD * nc;
            for (long c = 0; c < nc; ++c) {
                fb[c] = (c >= nz) ? a.f[F_VR][c] : 0.0;
                fb[nc + c] = a.f[F_VZ][c];
            }
        }
        /* density term: dv^{n+1/2}/db = dt F^n = (v^{n+1/2} - v^{n-1/2}) / b */
        for (long c = 0; c < nc; ++c) {
            double dvr = vr[c] - (n > 0 ? vhist[(long)(n - 1) * 2 * nc + c] : 0.0);
            double dvz = vz[c] - (n > 0 ? vhist[(long)(n - 1) * 2 * nc + nc + c] : 0.0);
            if (c >= nz) acc[G_BR * nc + c] += dvr / m.bvr[c] * a.f[F_VR][c];
            acc[G_BZ * nc + c] += dvz / m.bvz[c] * a.f[F_VZ][c];
        }

        velocity_step_T(&m, &a); /* Atau now holds dJ/dtau^n */
    }
    free(a.blk);
    model_free(&m);
    return 0;
}

/*
 * Chain rule from the node accumulators to per-cell gradients of J with
 * respect to lambda, mu and rho, and the per-cell pseudo-Hessians.
 * Cells inside the C-PML get zero.
 *   out [5][nr*nz]: g_lambda, g_mu, g_rho, H_lambda, H_mu
 */
int orc_finalize(const orc_grid *g, const double *vp, const double *vs, const double *rho,
                 const double *acc, double *out)
{
    model_t m;
    if (model_init(&m, g, vp, vs, rho)) return -1;
    const int nr = g->nr, nz = g->nz;
    long nc = m.ncell;
    double *gl = out, *gm = out + nc, *gr = out + 2 * nc, *hl = out + 3 * nc, *hm = out + 4 * nc;
    memset(out, 0, (size_t)5 * nc * sizeof(double));
    for (long c = 0; c < nc; ++c) {
        gl[c] = acc[G_LAM * nc + c];
        gm[c] = acc[G_MUNN * nc + c];
        hl[c] = acc[H_LAM * nc + c];
        hm[c] = acc[H_MUNN * nc + c];
    }
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nz; ++j) {
            long c = (long)i * nz + j;
            int jp = (j + 1 < nz) ? j + 1 : nz - 1;
            if (i >= 1) {
                /* harmonic mu at trz (i,j): d muh / d mu_q = muh^2 / (4 mu_q^2) */
                const long q[4] = {(long)(i - 1) * nz + j, (long)i * nz + j,
                                   (long)(i - 1) * nz + jp, (long)i * nz + jp};
                double mh = m.muh[c];
                for (int k = 0; k < 4; ++k) {
                    if (mh > 0.0) gm[q[k]] += mh * mh / (4.0 * m.mu[q[k]] * m.mu[q[k]]) *
                                              acc[G_MURZ * nc + c];
                    hm[q[k]] += 0.25 * acc[H_MURZ * nc + c];
                }
                /* buoyancy at v_r (i,j) = (1/rho[i-1,j] + 1/rho[i,j]) / 2 */
                const long p[2] = {(long)(i - 1) * nz + j, c};
                for (int k = 0; k < 2; ++k)
                    gr[p[k]] += -0.5 / (m.rho[p[k]] * m.rho[p[k]]) * acc[G_BR * nc + c];
            }
            /* buoyancy at v_z (i,j) = (1/rho[i,j] + 1/rho[i,j+1]) / 2 */
            const long p[2] = {c, (long)i * nz + jp};
            for (int k = 0; k < 2; ++k)
                gr[p[k]] += -0.5 / (m.rho[p[k]] * m.rho[p[k]]) * acc[G_BZ * nc + c];
        }
    /* the pseudo-Hessian shear term spreads over the 4 trz nodes of a cell;
     * the loop above gives each cell 1/4 of each of its (up to 4) nodes. */
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nz; ++j) {
            int inside = (i < nr - g->npml_r) && (j >= g->npml_z) && (j < nz - g->npml_z);
            if (!inside) {
                long c = (long)i * nz + j;
                gl[c] = gm[c] = gr[c] = hl[c] = hm[c] = 0.0;
            }
        }
    model_free(&m);
    return 0;
}
