/*
 * FP64 CPU oracle for the multiparameter (ln Vp, ln Ip) Born operator L and
 * its exact transpose L^T on a staggered grid.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. The product path never
 * calls it, and it shares no source with the CUDA path.
 *
 * What it computes (plain definition, no blocking or fusion):
 *   - Background / nonlinear modelling, Eq. (1): first-order system
 *       rho dv/dt + grad p = 0,  kappa div v + dp/dt = f_p,
 *     kappa = rho Vp^2, discretised with a Virieux-type staggered grid
 *     (p, kappa, rho at integer nodes, v_i at half nodes), leapfrog in time,
 *     staggered Taylor coefficients of order 2M, CPML in all padded strips.
 *   - Born modelling, Eq. (scattereqln): the exact Jacobian of the discrete
 *     scheme with respect to (dln Vp, dln Ip), through the map of Sec. 2:
 *     dln rho = dln Ip - dln Vp, dln kappa = dln Ip + dln Vp.
 *   - L^T: the exact transpose of discrete L under plain Euclidean inner
 *     products, obtained by transposing each sub-step of the Born recursion in
 *     reverse order (the discrete form of App. A, where the continuous adjoint
 *     and the cross-correlations of Eqs. (gradrho), (gradkappa) arise), and the
 *     chain rule of Sec. 3: g_Vp = g_kappa - g_rho, g_Ip = g_kappa + g_rho.
 *     The background wavefield is recomputed from full-state checkpoints.
 *   - The pseudo-Hessian diagonal of App. B.
 *
 * Readings where the paper is silent (discretisation, boundary, source, which
 * field is recorded) are fixed as follows:
 *   - values outside the padded array are zero, so D- = -(D+)^T exactly;
 *   - buoyancy at half node j along a direction = (1/rho_j + 1/rho_{j+1})/2
 *     (rho_{j+1} replicated at the array end); its derivative is exact;
 *   - model perturbations live on the interior only (zero in the pad);
 *   - the source adds dt*w[n]/cell_volume to p at step n (after the p update);
 *   - receivers record p (Born: dp) after step n: d[k][n] = p^{n+1}[rec_k];
 *   - CPML: quadratic damping d0 (dist/L)^2, d0 = -3 vmax ln(1e-4)/(2 L dx),
 *     alpha = pi f0 (1 - dist/L), kappa_pml = 1; dist is measured from the
 *     interface half node (interior edge - 1/2), so every interior node and
 *     every interface half node has no CPML memory.
 *   - optional free surface on the first interior row z_s (method of images):
 *     p = 0 on z_s; above it the rows are ghosts holding the odd mirror of p
 *     (p(z_s - j) = -p(z_s + j)) and the even mirror of v_z (half row
 *     z_s - 1 - j equals half row z_s + j), imposed after every pressure and
 *     velocity update; no CPML on top; the model rows above z_s are the mirror
 *     of those below it. L^T applies the transposes of these maps (the ghost
 *     values folded onto their mirrors, then cleared).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXM 4
#define ORC_PI 3.14159265358979323846

typedef struct {
    int ndim, nz, ny, nx, npml, order, nt;
    double dz, dy, dx, dt, f0, vmax;
    int free_surface;
} orc_cfg;

/* Direction index: 0 = z, 1 = y, 2 = x. */
typedef struct {
    int ndim, M;
    int n[3], ni[3], o[3];
    long s[3];
    long ncell;
    double h[3];
    double dt;
    double c[ORC_MAXM];
    int nd;          /* number of active directions */
    int dirs[3];     /* active directions */
    double *ai[3], *bi[3], *ah[3], *bh[3];
    double *kap, *rho, *bu[3];
    double cellvol;
    int fs;          /* free surface on row o[0] */
} grid;

/* ---------------------------------------------------------------- FD coeffs */

/* Staggered first-derivative coefficients of order 2M: the c_l that make
 * sum_l c_l (f(x+(l-1/2)h) - f(x-(l-1/2)h))/h exact for polynomials of degree
 * 2M, i.e. sum_l c_l (2l-1) = 1 and sum_l c_l (2l-1)^(2k-1) = 0, k = 2..M.
 * Solved by Gaussian elimination with partial pivoting. */
int orc_fd_coeffs(int order, double *c)
{
    int M = order / 2;
    if (order % 2 || M < 1 || M > ORC_MAXM) return 1;
    double A[ORC_MAXM][ORC_MAXM + 1];
    for (int k = 0; k < M; ++k) {
        for (int l = 0; l < M; ++l) A[k][l] = pow(2.0 * (l + 1) - 1.0, 2.0 * k + 1.0);
        A[k][M] = (k == 0) ? 1.0 : 0.0;
    }
    for (int col = 0; col < M; ++col) {
        int piv = col;
        for (int r = col + 1; r < M; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int j = 0; j <= M; ++j) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
        for (int r = 0; r < M; ++r) {
            if (r == col) continue;
            double f = A[r][col] / A[col][col];
            for (int j = col; j <= M; ++j) A[r][j] -= f * A[col][j];
        }
    }
    for (int l = 0; l < M; ++l) c[l] = A[l][M] / A[l][l];
    return 0;
}

/* ------------------------------------------------------------------ grid */

static void grid_free(grid *g)
{
    for (int d = 0; d < 3; ++d) {
        free(g->ai[d]); free(g->bi[d]); free(g->ah[d]); free(g->bh[d]); free(g->bu[d]);
        g->ai[d] = g->bi[d] = g->ah[d] = g->bh[d] = g->bu[d] = NULL;
    }
    free(g->kap); free(g->rho);
    g->kap = g->rho = NULL;
}

/* CPML damping profile at grid-unit distance `dist` beyond the interface. */
static void cpml_coef(double dist, double L, double d0, double alpha0, double dt,
                      double *a, double *b)
{
    if (dist <= 0.0) { *a = 0.0; *b = 0.0; return; }
    double r = dist / L;
    double d = d0 * r * r;
    double al = alpha0 * (1.0 - r);
    if (al < 0.0) al = 0.0;
    double bb = exp(-(d + al) * dt);
    *b = bb;
    *a = d * (bb - 1.0) / (d + al);
}

/* Pads the interior model by edge replication and derives kappa, buoyancy and
 * the CPML profiles. vp, rho are interior arrays [nz][ny][nx]. */
static int grid_init(grid *g, const orc_cfg *cfg, const double *vp, const double *rho_in)
{
    memset(g, 0, sizeof(*g));
    g->ndim = cfg->ndim;
    g->M = cfg->order / 2;
    if (orc_fd_coeffs(cfg->order, g->c)) return 1;
    if (cfg->ndim != 2 && cfg->ndim != 3) return 1;
    int P = cfg->npml;
    g->ni[0] = cfg->nz; g->ni[1] = (cfg->ndim == 3) ? cfg->ny : 1; g->ni[2] = cfg->nx;
    g->o[0] = P; g->o[1] = (cfg->ndim == 3) ? P : 0; g->o[2] = P;
    for (int d = 0; d < 3; ++d) g->n[d] = g->ni[d] + 2 * g->o[d];
    g->s[2] = 1; g->s[1] = g->n[2]; g->s[0] = (long)g->n[1] * g->n[2];
    g->ncell = (long)g->n[0] * g->n[1] * g->n[2];
    g->h[0] = cfg->dz; g->h[1] = cfg->dy; g->h[2] = cfg->dx;
    g->dt = cfg->dt;
    if (cfg->ndim == 2) { g->nd = 2; g->dirs[0] = 0; g->dirs[1] = 2; g->cellvol = cfg->dz * cfg->dx; }
    else { g->nd = 3; g->dirs[0] = 0; g->dirs[1] = 1; g->dirs[2] = 2; g->cellvol = cfg->dz * cfg->dy * cfg->dx; }

    g->fs = cfg->free_surface != 0;
    g->kap = (double *)malloc(sizeof(double) * g->ncell);
    g->rho = (double *)malloc(sizeof(double) * g->ncell);
    if (!g->kap || !g->rho) return 2;
    double vmax = cfg->vmax;
    int nyi = g->ni[1];
    for (int z = 0; z < g->n[0]; ++z)
        for (int y = 0; y < g->n[1]; ++y)
            for (int x = 0; x < g->n[2]; ++x) {
                int iz = z - g->o[0], iy = y - g->o[1], ix = x - g->o[2];
                if (iz < 0 && g->fs) iz = -iz;   /* mirror above the free surface */
                if (iz < 0) iz = 0; if (iz >= g->ni[0]) iz = g->ni[0] - 1;
                if (iy < 0) iy = 0; if (iy >= nyi) iy = nyi - 1;
                if (ix < 0) ix = 0; if (ix >= g->ni[2]) ix = g->ni[2] - 1;
                long k = ((long)iz * nyi + iy) * g->ni[2] + ix;
                long c = z * g->s[0] + y * g->s[1] + x;
                g->rho[c] = rho_in[k];
                g->kap[c] = rho_in[k] * vp[k] * vp[k];
            }
    if (vmax <= 0.0) {
        long nint = (long)g->ni[0] * nyi * g->ni[2];
        for (long k = 0; k < nint; ++k) if (vp[k] > vmax) vmax = vp[k];
    }
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        g->bu[d] = (double *)malloc(sizeof(double) * g->ncell);
        if (!g->bu[d]) return 2;
        for (int z = 0; z < g->n[0]; ++z)
            for (int y = 0; y < g->n[1]; ++y)
                for (int x = 0; x < g->n[2]; ++x) {
                    long c = z * g->s[0] + y * g->s[1] + x;
                    int i = (d == 0) ? z : (d == 1) ? y : x;
                    long cn = (i + 1 < g->n[d]) ? c + g->s[d] : c;
                    g->bu[d][c] = 0.5 * (1.0 / g->rho[c] + 1.0 / g->rho[cn]);
                }
        int N = g->n[d];
        g->ai[d] = (double *)calloc(N, sizeof(double));
        g->bi[d] = (double *)calloc(N, sizeof(double));
        g->ah[d] = (double *)calloc(N, sizeof(double));
        g->bh[d] = (double *)calloc(N, sizeof(double));
        if (!g->ai[d] || !g->bi[d] || !g->ah[d] || !g->bh[d]) return 2;
        double L = (double)P;
        double d0 = (P > 0) ? -3.0 * vmax * log(1e-4) / (2.0 * P * g->h[d]) : 0.0;
        double alpha0 = ORC_PI * cfg->f0;
        double x0 = g->o[d], x1 = g->o[d] + g->ni[d];
        for (int i = 0; i < N; ++i) {
            double di = fmax(0.0, fmax((x0 - 0.5) - i, i - (x1 - 0.5)));
            double dh = fmax(0.0, fmax((x0 - 0.5) - (i + 0.5), (i + 0.5) - (x1 - 0.5)));
            if (d == 0 && g->fs && i < x0) di = dh = 0.0;   /* no CPML above a free surface */
            cpml_coef(di, L, d0, alpha0, g->dt, &g->ai[d][i], &g->bi[d][i]);
            cpml_coef(dh, L, d0, alpha0, g->dt, &g->ah[d][i], &g->bh[d][i]);
        }
    }
    return 0;
}

static inline int coord(const grid *g, int d, int z, int y, int x)
{
    return (d == 0) ? z : (d == 1) ? y : x;
}

/* D+ f at half node (index i along d): sum_l c_l (f[i+l] - f[i+1-l]) / h. */
static inline double Dplus(const grid *g, const double *f, long c, int i, int d)
{
    double acc = 0.0;
    for (int l = 1; l <= g->M; ++l) {
        double a = (i + l < g->n[d]) ? f[c + l * g->s[d]] : 0.0;
        double b = (i + 1 - l >= 0) ? f[c + (1 - l) * g->s[d]] : 0.0;
        acc += g->c[l - 1] * (a - b);
    }
    return acc / g->h[d];
}

/* D- f at integer node (index i along d): sum_l c_l (f[i+l-1] - f[i-l]) / h. */
static inline double Dminus(const grid *g, const double *f, long c, int i, int d)
{
    double acc = 0.0;
    for (int l = 1; l <= g->M; ++l) {
        double a = (i + l - 1 < g->n[d]) ? f[c + (l - 1) * g->s[d]] : 0.0;
        double b = (i - l >= 0) ? f[c - l * g->s[d]] : 0.0;
        acc += g->c[l - 1] * (a - b);
    }
    return acc / g->h[d];
}

#define FOR_CELLS(g) \
    for (int z = 0; z < (g)->n[0]; ++z) \
        for (int y = 0; y < (g)->n[1]; ++y) \
            for (int x = 0; x < (g)->n[2]; ++x)
#define CELL(g) ((long)z * (g)->s[0] + (long)y * (g)->s[1] + x)

/* ------------------------------------------------------------ wave state */

typedef struct {
    double *p, *v[3], *psip[3], *psiv[3];
} state;

static int state_alloc(const grid *g, state *st)
{
    memset(st, 0, sizeof(*st));
    st->p = (double *)calloc(g->ncell, sizeof(double));
    if (!st->p) return 2;
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        st->v[d] = (double *)calloc(g->ncell, sizeof(double));
        st->psip[d] = (double *)calloc(g->ncell, sizeof(double));
        st->psiv[d] = (double *)calloc(g->ncell, sizeof(double));
        if (!st->v[d] || !st->psip[d] || !st->psiv[d]) return 2;
    }
    return 0;
}

static void state_free(state *st)
{
    free(st->p);
    for (int d = 0; d < 3; ++d) { free(st->v[d]); free(st->psip[d]); free(st->psiv[d]); }
    memset(st, 0, sizeof(*st));
}

static void state_zero(const grid *g, state *st)
{
    memset(st->p, 0, sizeof(double) * g->ncell);
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        memset(st->v[d], 0, sizeof(double) * g->ncell);
        memset(st->psip[d], 0, sizeof(double) * g->ncell);
        memset(st->psiv[d], 0, sizeof(double) * g->ncell);
    }
}

static void state_copy(const grid *g, state *dst, const state *src)
{
    memcpy(dst->p, src->p, sizeof(double) * g->ncell);
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        memcpy(dst->v[d], src->v[d], sizeof(double) * g->ncell);
        memcpy(dst->psip[d], src->psip[d], sizeof(double) * g->ncell);
        memcpy(dst->psiv[d], src->psiv[d], sizeof(double) * g->ncell);
    }
}

/* ---------------------------------------------------- free surface maps */

/* E_v: ghost half rows of v_z take the even mirror, v_z(z_s-1-j) = v_z(z_s+j). */
static void fs_mirror_v(const grid *g, double *vz)
{
    if (!g->fs) return;
    int zs = g->o[0];
    for (int z = 0; z < zs; ++z) {
        int zm = 2 * zs - 1 - z;
        if (zm >= g->n[0]) { memset(vz + z * g->s[0], 0, sizeof(double) * g->s[0]); continue; }
        memcpy(vz + z * g->s[0], vz + zm * g->s[0], sizeof(double) * g->s[0]);
    }
}

/* E_p: p(z_s) = 0 and ghost rows the odd mirror, p(z_s-j) = -p(z_s+j). */
static void fs_mirror_p(const grid *g, double *p)
{
    if (!g->fs) return;
    int zs = g->o[0];
    memset(p + zs * g->s[0], 0, sizeof(double) * g->s[0]);
    for (int z = 0; z < zs; ++z) {
        int zm = 2 * zs - z;
        for (long c = 0; c < g->s[0]; ++c) p[z * g->s[0] + c] = (zm < g->n[0]) ? -p[zm * g->s[0] + c] : 0.0;
    }
}

/* E_v^T: each ghost half row's adjoint added onto its mirror, then cleared. */
static void fs_fold_v(const grid *g, double *lvz)
{
    if (!g->fs) return;
    int zs = g->o[0];
    for (int z = 0; z < zs; ++z) {
        int zm = 2 * zs - 1 - z;
        if (zm < g->n[0])
            for (long c = 0; c < g->s[0]; ++c) lvz[zm * g->s[0] + c] += lvz[z * g->s[0] + c];
        memset(lvz + z * g->s[0], 0, sizeof(double) * g->s[0]);
    }
}

/* E_p^T: each ghost row's adjoint subtracted from its mirror, then the ghost
 * rows and the surface row cleared. */
static void fs_fold_p(const grid *g, double *lp)
{
    if (!g->fs) return;
    int zs = g->o[0];
    for (int z = 0; z < zs; ++z) {
        int zm = 2 * zs - z;
        if (zm < g->n[0])
            for (long c = 0; c < g->s[0]; ++c) lp[zm * g->s[0] + c] -= lp[z * g->s[0] + c];
        memset(lp + z * g->s[0], 0, sizeof(double) * g->s[0]);
    }
    memset(lp + zs * g->s[0], 0, sizeof(double) * g->s[0]);
}

/* One time step of Eq. (1) without the source: v^{n+1/2} from p^n, then
 * p^{n+1} from v^{n+1/2}, each with its CPML memory. Optionally returns the
 * terms the Born sources multiply: G[d] = D+_d p^n + psi_p (half nodes) and
 * Q = sum_d (D-_d v_d + psi_v) (integer nodes). */
static void fwd_step(const grid *g, state *st, double **G, double *Q)
{
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            double dp = Dplus(g, st->p, c, i, d);
            st->psip[d][c] = g->bh[d][i] * st->psip[d][c] + g->ah[d][i] * dp;
            double gg = dp + st->psip[d][c];
            if (G) G[d][c] = gg;
            st->v[d][c] -= g->dt * g->bu[d][c] * gg;
        }
    }
    fs_mirror_v(g, st->v[0]);
    FOR_CELLS(g) {
        long c = CELL(g);
        double qq = 0.0;
        for (int k = 0; k < g->nd; ++k) {
            int d = g->dirs[k];
            int i = coord(g, d, z, y, x);
            double dv = Dminus(g, st->v[d], c, i, d);
            st->psiv[d][c] = g->bi[d][i] * st->psiv[d][c] + g->ai[d][i] * dv;
            qq += dv + st->psiv[d][c];
        }
        if (Q) Q[c] = qq;
        st->p[c] -= g->dt * g->kap[c] * qq;
    }
}

/* One step of the linearised (Born) recursion, Eq. (scattereqln): the
 * scattered state advances in the background medium and is driven by
 *   -dt * dbu_d * G_d   (velocity, from dln rho through the buoyancy) and
 *   -dt * dkap * Q      (pressure, from dln kappa). */
static void born_step(const grid *g, state *ds, double *const *G, const double *Q,
                      double *const *dbu, const double *dkap)
{
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            double dp = Dplus(g, ds->p, c, i, d);
            ds->psip[d][c] = g->bh[d][i] * ds->psip[d][c] + g->ah[d][i] * dp;
            ds->v[d][c] -= g->dt * (g->bu[d][c] * (dp + ds->psip[d][c]) + dbu[d][c] * G[d][c]);
        }
    }
    fs_mirror_v(g, ds->v[0]);
    FOR_CELLS(g) {
        long c = CELL(g);
        double qq = 0.0;
        for (int k = 0; k < g->nd; ++k) {
            int d = g->dirs[k];
            int i = coord(g, d, z, y, x);
            double dv = Dminus(g, ds->v[d], c, i, d);
            ds->psiv[d][c] = g->bi[d][i] * ds->psiv[d][c] + g->ai[d][i] * dv;
            qq += dv + ds->psiv[d][c];
        }
        ds->p[c] -= g->dt * (g->kap[c] * qq + dkap[c] * Q[c]);
    }
    fs_mirror_p(g, ds->p);
}

/* Transpose of born_step (sub-steps reversed, each transposed), accumulating
 * the gradient w.r.t. dln kappa (gk) and w.r.t. r = dln rho / rho (gr). The
 * forward sub-steps are, per direction d:
 *   S1: psip_d <- bh psip_d + ah D+ p
 *   S2: v_d    <- v_d - dt bu (D+ p + psip_d) - dt dbu_d(r) G_d
 *   S3: psiv_d <- bi psiv_d + ai D- v_d
 *   S4: p      <- p - dt kap sum_d (D- v_d + psiv_d) - dt kap dlnk Q
 * with (D-)^T = -D+ and (D+)^T = -D-. */
static void adj_step(const grid *g, state *ls, double *const *G, const double *Q,
                     double *gk, double *gr, double *t1, double *t2)
{
    double dt = g->dt;
    /* E_p^T (the Born step ends with E_p) */
    fs_fold_p(g, ls->p);
    /* S4^T */
    FOR_CELLS(g) {
        long c = CELL(g);
        gk[c] += -dt * g->kap[c] * Q[c] * ls->p[c];
        t1[c] = g->kap[c] * ls->p[c];
    }
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            ls->psiv[d][c] += -dt * t1[c];
            ls->v[d][c] += dt * Dplus(g, t1, c, i, d);
        }
    }
    /* S3^T */
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            t2[c] = g->ai[d][coord(g, d, z, y, x)] * ls->psiv[d][c];
        }
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            ls->v[d][c] -= Dplus(g, t2, c, i, d);
            ls->psiv[d][c] *= g->bi[d][i];
        }
    }
    /* E_v^T (E_v follows the velocity update S2) */
    fs_fold_v(g, ls->v[0]);
    /* S2^T then S1^T, per direction */
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            double P = G[d][c] * ls->v[d][c];
            gr[c] += 0.5 * dt * P;
            if (i + 1 < g->n[d]) gr[c + g->s[d]] += 0.5 * dt * P;
            t2[c] = g->bu[d][c] * ls->v[d][c];
            ls->psip[d][c] += -dt * t2[c];
        }
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            ls->p[c] += dt * Dminus(g, t2, c, i, d);
        }
        FOR_CELLS(g) {
            long c = CELL(g);
            t2[c] = g->ah[d][coord(g, d, z, y, x)] * ls->psip[d][c];
        }
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            ls->p[c] -= Dminus(g, t2, c, i, d);
            ls->psip[d][c] *= g->bh[d][i];
        }
    }
}

/* ------------------------------------------------------------- helpers */

static long pad_index(const grid *g, long k)
{
    int nx = g->ni[2], ny = g->ni[1];
    long ix = k % nx;
    long iy = (k / nx) % ny;
    long iz = k / ((long)nx * ny);
    return (iz + g->o[0]) * g->s[0] + (iy + g->o[1]) * g->s[1] + (ix + g->o[2]);
}

static long nint_of(const grid *g) { return (long)g->ni[0] * g->ni[1] * g->ni[2]; }

static int check_geom(const grid *g, int nshot, const int *src_ptr, const int *src_idx,
                      const int *rec_ptr, const int *rec_idx)
{
    long nint = nint_of(g);
    for (int s = 0; s < nshot; ++s) {
        if (src_ptr[s + 1] < src_ptr[s] || rec_ptr[s + 1] < rec_ptr[s]) return 3;
        for (int j = src_ptr[s]; j < src_ptr[s + 1]; ++j)
            if (src_idx[j] < 0 || src_idx[j] >= nint) return 3;
        for (int j = rec_ptr[s]; j < rec_ptr[s + 1]; ++j)
            if (rec_idx[j] < 0 || rec_idx[j] >= nint) return 3;
    }
    return 0;
}

static void inject(const grid *g, double *p, int s, int n, const int *src_ptr,
                   const int *src_idx, const double *wav, int nt, int wav_per_shot)
{
    double w = wav[(wav_per_shot ? (long)s * nt : 0) + n];
    for (int j = src_ptr[s]; j < src_ptr[s + 1]; ++j)
        p[pad_index(g, src_idx[j])] += g->dt * w / g->cellvol;
}

/* ----------------------------------------------------------- public API */

/* Nonlinear modelling: records p^{n+1} at the receivers, d[rec][n]. */
int orc_model(const orc_cfg *cfg, const double *vp, const double *rho, const double *wav,
              int wav_per_shot, int nshot, const int *src_ptr, const int *src_idx,
              const int *rec_ptr, const int *rec_idx, double *d)
{
    grid g;
    int err = grid_init(&g, cfg, vp, rho);
    if (!err) err = check_geom(&g, nshot, src_ptr, src_idx, rec_ptr, rec_idx);
    if (err) { grid_free(&g); return err; }
    int nt = cfg->nt;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int s = 0; s < nshot; ++s) {
        state st;
        if (state_alloc(&g, &st)) { state_free(&st); fail |= 2; continue; }
        for (int n = 0; n < nt; ++n) {
            fwd_step(&g, &st, NULL, NULL);
            inject(&g, st.p, s, n, src_ptr, src_idx, wav, nt, wav_per_shot);
            fs_mirror_p(&g, st.p);
            for (int k = rec_ptr[s]; k < rec_ptr[s + 1]; ++k)
                d[(long)k * nt + n] = st.p[pad_index(&g, rec_idx[k])];
        }
        state_free(&st);
    }
    grid_free(&g);
    return fail;
}

/* Pressure snapshot p^{nsnap} (padded grid) of shot 0, for propagation tests. */
int orc_snapshot(const orc_cfg *cfg, const double *vp, const double *rho, const double *wav,
                 const int *src_ptr, const int *src_idx, int nsnap, double *p_out)
{
    grid g;
    int err = grid_init(&g, cfg, vp, rho);
    if (err) { grid_free(&g); return err; }
    state st;
    if (state_alloc(&g, &st)) { state_free(&st); grid_free(&g); return 2; }
    for (int n = 0; n < nsnap; ++n) {
        fwd_step(&g, &st, NULL, NULL);
        inject(&g, st.p, 0, n, src_ptr, src_idx, wav, cfg->nt, 0);
        fs_mirror_p(&g, st.p);
    }
    memcpy(p_out, st.p, sizeof(double) * g.ncell);
    state_free(&st);
    grid_free(&g);
    return 0;
}

/* Perturbation map of Sec. 2 on the padded grid: dkap = kap * (dlnVp + dlnIp),
 * r = (dlnIp - dlnVp) / rho, and dbu_d = -(r_j + r_{j+1})/2 at half nodes. */
static int perturbation(const grid *g, const double *dm, double *dkap, double *r, double **dbu)
{
    long nint = nint_of(g);
    memset(dkap, 0, sizeof(double) * g->ncell);
    memset(r, 0, sizeof(double) * g->ncell);
    for (long k = 0; k < nint; ++k) {
        long c = pad_index(g, k);
        double m1 = dm[k], m2 = dm[nint + k];
        dkap[c] = g->kap[c] * (m2 + m1);
        r[c] = (m2 - m1) / g->rho[c];
    }
    for (int q = 0; q < g->nd; ++q) {
        int d = g->dirs[q];
        FOR_CELLS(g) {
            long c = CELL(g);
            int i = coord(g, d, z, y, x);
            double rn = (i + 1 < g->n[d]) ? r[c + g->s[d]] : 0.0;
            dbu[d][c] = -0.5 * (r[c] + rn);
        }
    }
    return 0;
}

/* Born modelling d = L dm; dm = [2][nint] (dln Vp, dln Ip), d = [rec][nt]. */
int orc_born(const orc_cfg *cfg, const double *vp, const double *rho, const double *wav,
             int wav_per_shot, int nshot, const int *src_ptr, const int *src_idx,
             const int *rec_ptr, const int *rec_idx, const double *dm, double *d)
{
    grid g;
    int err = grid_init(&g, cfg, vp, rho);
    if (!err) err = check_geom(&g, nshot, src_ptr, src_idx, rec_ptr, rec_idx);
    if (err) { grid_free(&g); return err; }
    double *dkap = (double *)malloc(sizeof(double) * g.ncell);
    double *r = (double *)malloc(sizeof(double) * g.ncell);
    double *dbu[3] = {0, 0, 0};
    for (int q = 0; q < g.nd; ++q) dbu[g.dirs[q]] = (double *)malloc(sizeof(double) * g.ncell);
    perturbation(&g, dm, dkap, r, dbu);
    int nt = cfg->nt;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int s = 0; s < nshot; ++s) {
        state st, ds;
        double *G[3] = {0, 0, 0};
        double *Q = (double *)malloc(sizeof(double) * g.ncell);
        int e = state_alloc(&g, &st) | state_alloc(&g, &ds) | (Q == NULL);
        for (int q = 0; q < g.nd; ++q) {
            G[g.dirs[q]] = (double *)malloc(sizeof(double) * g.ncell);
            if (!G[g.dirs[q]]) e = 1;
        }
        if (!e) {
            for (int n = 0; n < nt; ++n) {
                fwd_step(&g, &st, G, Q);
                inject(&g, st.p, s, n, src_ptr, src_idx, wav, nt, wav_per_shot);
                fs_mirror_p(&g, st.p);
                born_step(&g, &ds, G, Q, dbu, dkap);
                for (int k = rec_ptr[s]; k < rec_ptr[s + 1]; ++k)
                    d[(long)k * nt + n] = ds.p[pad_index(&g, rec_idx[k])];
            }
        } else {
            fail |= 2;
        }
        for (int q = 0; q < 3; ++q) free(G[q]);
        free(Q);
        state_free(&st);
        state_free(&ds);
    }
    free(dkap); free(r);
    for (int q = 0; q < 3; ++q) free(dbu[q]);
    grid_free(&g);
    return fail;
}

/* L^T: g = [2][nint] (dln Vp, dln Ip) from data d = [rec][nt]. graw, if not
 * NULL, receives [2][nint] = (g_kappa, g_rho) before the chain rule. The
 * background is recomputed segment by segment from full-state checkpoints
 * taken every K = ceil(sqrt(nt)) steps. */
int orc_adjoint(const orc_cfg *cfg, const double *vp, const double *rho, const double *wav,
                int wav_per_shot, int nshot, const int *src_ptr, const int *src_idx,
                const int *rec_ptr, const int *rec_idx, const double *d, double *gout,
                double *graw)
{
    grid g;
    int err = grid_init(&g, cfg, vp, rho);
    if (!err) err = check_geom(&g, nshot, src_ptr, src_idx, rec_ptr, rec_idx);
    if (err) { grid_free(&g); return err; }
    int nt = cfg->nt;
    int K = (int)ceil(sqrt((double)nt));
    if (K < 1) K = 1;
    int nseg = (nt + K - 1) / K;
    long nc = g.ncell;
    double *gk_all = (double *)calloc((size_t)nshot * nc, sizeof(double));
    double *gr_all = (double *)calloc((size_t)nshot * nc, sizeof(double));
    if (!gk_all || !gr_all) { free(gk_all); free(gr_all); grid_free(&g); return 2; }
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int s = 0; s < nshot; ++s) {
        state st, ls;
        state *ck = (state *)calloc(nseg, sizeof(state));
        double *Gs = (double *)malloc(sizeof(double) * (size_t)K * 3 * nc);
        double *Qs = (double *)malloc(sizeof(double) * (size_t)K * nc);
        double *t1 = (double *)malloc(sizeof(double) * nc);
        double *t2 = (double *)malloc(sizeof(double) * nc);
        int e = state_alloc(&g, &st) | state_alloc(&g, &ls);
        if (!ck || !Gs || !Qs || !t1 || !t2) e = 1;
        for (int j = 0; j < nseg && !e; ++j) e |= state_alloc(&g, &ck[j]);
        if (!e) {
            double *gk = gk_all + (size_t)s * nc, *gr = gr_all + (size_t)s * nc;
            /* forward pass: checkpoint the state at the start of each segment */
            for (int n = 0; n < nt; ++n) {
                if (n % K == 0) state_copy(&g, &ck[n / K], &st);
                fwd_step(&g, &st, NULL, NULL);
                inject(&g, st.p, s, n, src_ptr, src_idx, wav, nt, wav_per_shot);
                fs_mirror_p(&g, st.p);
            }
            /* reverse pass */
            for (int j = nseg - 1; j >= 0; --j) {
                int n0 = j * K, n1 = (n0 + K < nt) ? n0 + K : nt;
                state_copy(&g, &st, &ck[j]);
                for (int n = n0; n < n1; ++n) {
                    double *G[3] = {0, 0, 0};
                    for (int q = 0; q < g.nd; ++q)
                        G[g.dirs[q]] = Gs + ((size_t)(n - n0) * 3 + g.dirs[q]) * nc;
                    fwd_step(&g, &st, G, Qs + (size_t)(n - n0) * nc);
                    inject(&g, st.p, s, n, src_ptr, src_idx, wav, nt, wav_per_shot);
                    fs_mirror_p(&g, st.p);
                }
                for (int n = n1 - 1; n >= n0; --n) {
                    double *G[3] = {0, 0, 0};
                    for (int q = 0; q < g.nd; ++q)
                        G[g.dirs[q]] = Gs + ((size_t)(n - n0) * 3 + g.dirs[q]) * nc;
                    /* S5^T: receiver injection */
                    for (int k = rec_ptr[s]; k < rec_ptr[s + 1]; ++k)
                        ls.p[pad_index(&g, rec_idx[k])] += d[(long)k * nt + n];
                    adj_step(&g, &ls, G, Qs + (size_t)(n - n0) * nc, gk, gr, t1, t2);
                }
            }
        } else {
            fail |= 2;
        }
        for (int j = 0; j < nseg && ck; ++j) state_free(&ck[j]);
        free(ck); free(Gs); free(Qs); free(t1); free(t2);
        state_free(&st); state_free(&ls);
    }
    if (!fail) {
        long nint = nint_of(&g);
        for (long k = 0; k < nint; ++k) {
            long c = pad_index(&g, k);
            double sk = 0.0, sr = 0.0;
            for (int s = 0; s < nshot; ++s) {
                sk += gk_all[(size_t)s * nc + c];
                sr += gr_all[(size_t)s * nc + c];
            }
            sr /= g.rho[c];  /* gradient w.r.t. dln rho = (d/dr) / rho */
            gout[k] = sk - sr;          /* dln Vp */
            gout[nint + k] = sk + sr;   /* dln Ip */
            if (graw) { graw[k] = sk; graw[nint + k] = sr; }
        }
    }
    free(gk_all); free(gr_all);
    grid_free(&g);
    return fail;
}

/* Pseudo-Hessian diagonal of App. B, summed over shots:
 *   H = dt sum_n [ rho^2 sum_d (|bu G_d|^2 at the two half nodes around the
 *       node, averaged) + kap^2 Q^2 ],
 * with the discrete dt v = -bu G and div v = Q of the scheme. Returned on the
 * interior, [nint]; the same array serves dln Vp and dln Ip. */
int orc_pseudo_hessian(const orc_cfg *cfg, const double *vp, const double *rho,
                       const double *wav, int wav_per_shot, int nshot, const int *src_ptr,
                       const int *src_idx, double *h)
{
    grid g;
    int err = grid_init(&g, cfg, vp, rho);
    if (err) { grid_free(&g); return err; }
    long nc = g.ncell, nint = nint_of(&g);
    int nt = cfg->nt;
    double *hall = (double *)calloc((size_t)nshot * nc, sizeof(double));
    if (!hall) { grid_free(&g); return 2; }
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int s = 0; s < nshot; ++s) {
        state st;
        double *G[3] = {0, 0, 0};
        double *Q = (double *)malloc(sizeof(double) * nc);
        int e = state_alloc(&g, &st) | (Q == NULL);
        for (int q = 0; q < g.nd; ++q) {
            G[g.dirs[q]] = (double *)malloc(sizeof(double) * nc);
            if (!G[g.dirs[q]]) e = 1;
        }
        if (!e) {
            double *hs = hall + (size_t)s * nc;
            for (int n = 0; n < nt; ++n) {
                fwd_step(&g, &st, G, Q);
                inject(&g, st.p, s, n, src_ptr, src_idx, wav, nt, wav_per_shot);
                fs_mirror_p(&g, st.p);
                FOR_CELLS(&g) {
                    long c = CELL(&g);
                    double hr = 0.0;
                    for (int q = 0; q < g.nd; ++q) {
                        int d = g.dirs[q];
                        int i = coord(&g, d, z, y, x);
                        double a = g.bu[d][c] * G[d][c];
                        double b = (i > 0) ? g.bu[d][c - g.s[d]] * G[d][c - g.s[d]] : 0.0;
                        hr += 0.5 * (a * a + b * b);
                    }
                    hs[c] += g.dt * (g.rho[c] * g.rho[c] * hr + g.kap[c] * g.kap[c] * Q[c] * Q[c]);
                }
            }
        } else {
            fail |= 2;
        }
        for (int q = 0; q < 3; ++q) free(G[q]);
        free(Q);
        state_free(&st);
    }
    if (!fail) {
        for (long k = 0; k < nint; ++k) {
            long c = pad_index(&g, k);
            double acc = 0.0;
            for (int s = 0; s < nshot; ++s) acc += hall[(size_t)s * nc + c];
            h[k] = acc;
        }
    }
    free(hall);
    grid_free(&g);
    return fail;
}

/* Threads the OpenMP runtime will use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
