/*
 * Plain FP64 CPU oracle for the second-order (quadratic) upwind-DG sweep on
 * tetrahedra.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; it shares no code, header or helper with the library.
 * Compiled with -ffp-contract=off.
 *
 * The paper runs first-, second- and third-order finite-element sweeps
 * (Sec. 3.6, the orders of Fig. 5 and Table 3); this file is
 * the second-order element on tetrahedra, written as the plain definition:
 *
 *   basis: quadratic Lagrange, ten nodes per cell, in this order:
 *     i = 0..3   the cell's vertices (local order of tets[c]),
 *                phi_v = lambda_v (2 lambda_v - 1);
 *     i = 4..9   the midpoints of the edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3),
 *                phi_(a,b) = 4 lambda_a lambda_b;
 *   local system per (cell, direction, group), the upwind-DG weak form of
 *   Eq. (1) integrated back by parts (as for the linear element):
 *
 *     sum_j [ int_K phi_i Omega.grad phi_j + sigma_t int_K phi_i phi_j
 *             + sum_{f inflow} |Omega.n_f| int_f phi_i phi_j ] psi_j
 *       = int_K phi_i (q + Omega.S1) + sum_{f inflow} |Omega.n_f| int_f phi_i psi_up
 *
 *   with q and S1 the quadratic interpolants of their nodal values, and
 *   psi_up the upwind cell's quadratic field evaluated at the same physical
 *   point (conforming trace), or on a boundary inflow face the prescribed
 *   field psi_bc of the cell itself (NULL: vacuum).
 *
 * Every integral is evaluated by a collapsed-coordinate (Duffy) Gauss-Legendre
 * product rule with 4 points per axis: exact for the polynomial degrees that
 * occur (at most 4 on the cell and on a face).  The local 10 x 10 system is
 * solved by Gaussian elimination with partial pivoting; cells are visited in
 * (t-level, cell id) order, all groups per visit (Algorithm 1).
 *
 * Geometry (volumes, basis gradients = grad lambda, area-weighted outward face
 * normals N_f, neighbours) and the face classification / t-levels come from
 * the first-order oracle's functions, called by the Python layer.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_NOMEM 5
#define ORA_ERR_SINGULAR 9

#define NB 10 /* nodes per cell */
#define NQ 4  /* Gauss-Legendre points per collapsed axis */

typedef struct {
    int64_t nc;
    int32_t G;
    int32_t D;
    const double *xyz;        /* [nv][3] */
    const int32_t *tets;      /* [nc][4] */
    const double *vol;        /* [nc] */
    const double *grad;       /* [nc][4][3]  grad lambda_k */
    const double *normal;     /* [nc][4][3]  area-weighted outward normal of face f (opposite vertex f) */
    const int32_t *nbr;       /* [nc][4] */
    const double *omega;      /* [D][3] */
    const double *w;          /* [D] */
    const uint8_t *inflow;    /* [D][nc] bit f: face f is inflow */
    const int32_t *level;     /* [D][nc] */
    const int32_t *material;  /* [nc] */
    const double *sigma_t;    /* [M][G] */
    const double *S1;         /* [nc][G][10][3] or NULL: extra angular source Omega.S1(x) */
    const double *psi_bc;     /* [nc][G][10] or NULL: inflow field on boundary inflow faces */
} ora2_problem;

static const int EDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

/* Gauss-Legendre on [0, 1], NQ points (Newton on P_n, three-term recurrence). */
static void gl01(double *x, double *w)
{
    const int n = NQ;
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  /* 2/((1-z^2)P'^2) on [-1,1], halved */
    }
}

/* The ten basis functions at barycentric coordinates l[4]. */
static void basis(const double l[4], double phi[NB])
{
    for (int v = 0; v < 4; ++v) phi[v] = l[v] * (2.0 * l[v] - 1.0);
    for (int e = 0; e < 6; ++e) phi[4 + e] = 4.0 * l[EDGE[e][0]] * l[EDGE[e][1]];
}

/* d phi_i / d lambda_k at l: dphi[i][k]. */
static void basis_dl(const double l[4], double dphi[NB][4])
{
    memset(dphi, 0, sizeof(double) * NB * 4);
    for (int v = 0; v < 4; ++v) dphi[v][v] = 4.0 * l[v] - 1.0;
    for (int e = 0; e < 6; ++e) {
        const int a = EDGE[e][0], b = EDGE[e][1];
        dphi[4 + e][a] = 4.0 * l[b];
        dphi[4 + e][b] = 4.0 * l[a];
    }
}

/* Cell rule: barycentrics [NQ^3][4] and weights summing to 1 (times V gives
 * the integral over the cell).  xi1 = u, xi2 = v (1 - u), xi3 = t (1 - u)(1 - v),
 * Jacobian (1 - u)^2 (1 - v), reference volume 1/6. */
static void cell_rule(double lq[NQ * NQ * NQ][4], double wq[NQ * NQ * NQ])
{
    double x[NQ], w[NQ];
    gl01(x, w);
    int k = 0;
    for (int i = 0; i < NQ; ++i)
        for (int j = 0; j < NQ; ++j)
            for (int m = 0; m < NQ; ++m, ++k) {
                const double u = x[i], v = x[j], t = x[m];
                const double x1 = u, x2 = v * (1.0 - u), x3 = t * (1.0 - u) * (1.0 - v);
                lq[k][1] = x1;
                lq[k][2] = x2;
                lq[k][3] = x3;
                lq[k][0] = 1.0 - x1 - x2 - x3;
                wq[k] = 6.0 * w[i] * w[j] * w[m] * (1.0 - u) * (1.0 - u) * (1.0 - v);
            }
}

/* Triangle rule: (eta1, eta2) with eta1 = s, eta2 = t (1 - s), Jacobian (1 - s),
 * reference area 1/2; weights summing to 1 (times the face area). */
static void tri_rule(double eq[NQ * NQ][2], double wq[NQ * NQ])
{
    double x[NQ], w[NQ];
    gl01(x, w);
    int k = 0;
    for (int i = 0; i < NQ; ++i)
        for (int j = 0; j < NQ; ++j, ++k) {
            eq[k][0] = x[i];
            eq[k][1] = x[j] * (1.0 - x[i]);
            wq[k] = 2.0 * w[i] * w[j] * (1.0 - x[i]);
        }
}

/* Barycentric coordinates of physical point x in cell c: lambda_k(x) = 1/4 + grad lambda_k . (x - centroid). */
static void bary(const ora2_problem *P, int64_t c, const double x[3], double l[4])
{
    const int32_t *t = P->tets + 4 * c;
    double xc[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i)
        for (int d = 0; d < 3; ++d) xc[d] += 0.25 * P->xyz[3 * t[i] + d];
    const double *gr = P->grad + 12 * c;
    for (int k = 0; k < 4; ++k)
        l[k] = 0.25 + ((gr[3 * k] * (x[0] - xc[0]) + gr[3 * k + 1] * (x[1] - xc[1])) + gr[3 * k + 2] * (x[2] - xc[2]));
}

/* Reference integrals int_K phi_i / V by the cell rule (for the integrated flux and the tests). */
int ora2_basis_integrals(double *out)
{
    double lq[NQ * NQ * NQ][4], wq[NQ * NQ * NQ];
    cell_rule(lq, wq);
    for (int i = 0; i < NB; ++i) out[i] = 0.0;
    for (int k = 0; k < NQ * NQ * NQ; ++k) {
        double phi[NB];
        basis(lq[k], phi);
        for (int i = 0; i < NB; ++i) out[i] += wq[k] * phi[i];
    }
    return ORA_OK;
}

/* Reference mass matrix int_K phi_i phi_j / V by the cell rule. */
int ora2_mass(double *out)
{
    double lq[NQ * NQ * NQ][4], wq[NQ * NQ * NQ];
    cell_rule(lq, wq);
    memset(out, 0, sizeof(double) * NB * NB);
    for (int k = 0; k < NQ * NQ * NQ; ++k) {
        double phi[NB];
        basis(lq[k], phi);
        for (int i = 0; i < NB; ++i)
            for (int j = 0; j < NB; ++j) out[i * NB + j] += wq[k] * phi[i] * phi[j];
    }
    return ORA_OK;
}

static int lu_solve(double A[NB][NB], double b[NB], double x[NB])
{
    for (int k = 0; k < NB; ++k) {
        int p = k;
        for (int i = k + 1; i < NB; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == 0.0) return ORA_ERR_SINGULAR;
        if (p != k) {
            for (int j = 0; j < NB; ++j) { double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < NB; ++i) {
            double m = A[i][k] / A[k][k];
            for (int j = k; j < NB; ++j) A[i][j] -= m * A[k][j];
            b[i] -= m * b[k];
        }
    }
    for (int i = NB - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < NB; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return ORA_OK;
}

/* Sweep one direction for all groups: psi [nc][G][10]; q [nc][G][10] is the
 * isotropic angular source per steradian at the nodes. */
int ora2_sweep_direction(const ora2_problem *P, int a, const double *q, double *psi)
{
    const int64_t nc = P->nc;
    const int G = P->G;
    const uint8_t *mask = P->inflow + (size_t)a * nc;
    const int32_t *lev = P->level + (size_t)a * nc;
    const double *O = P->omega + 3 * a;
    static double lq[NQ * NQ * NQ][4], wq[NQ * NQ * NQ], eq[NQ * NQ][2], we[NQ * NQ];
    static int rules = 0;
#ifdef _OPENMP
#pragma omp critical(ora2_rules)
#endif
    if (!rules) {
        cell_rule(lq, wq);
        tri_rule(eq, we);
        rules = 1;
    }
    int32_t maxlev = 0;
    for (int64_t c = 0; c < nc; ++c) if (lev[c] > maxlev) maxlev = lev[c];
    int64_t *start = calloc((size_t)maxlev + 2, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    if (!start || !order) { free(start); free(order); return ORA_ERR_NOMEM; }
    for (int64_t c = 0; c < nc; ++c) start[lev[c] + 1]++;
    for (int32_t l = 0; l <= maxlev; ++l) start[l + 1] += start[l];
    for (int64_t c = 0; c < nc; ++c) order[start[lev[c]]++] = c;
    free(start);

    int status = ORA_OK;
    for (int64_t idx = 0; idx < nc && status == ORA_OK; ++idx) {
        const int64_t c = order[idx];
        const double V = P->vol[c];
        const double *gr = P->grad + 12 * c;
        double og[4]; /* Omega . grad lambda_k */
        for (int k = 0; k < 4; ++k) og[k] = (O[0] * gr[3 * k] + O[1] * gr[3 * k + 1]) + O[2] * gr[3 * k + 2];
        /* group-independent parts: streaming matrix and mass matrix over the cell */
        double Kc[NB][NB], Mc[NB][NB];
        memset(Kc, 0, sizeof(Kc));
        memset(Mc, 0, sizeof(Mc));
        for (int k = 0; k < NQ * NQ * NQ; ++k) {
            double phi[NB], dphi[NB][4];
            basis(lq[k], phi);
            basis_dl(lq[k], dphi);
            const double W = V * wq[k];
            for (int j = 0; j < NB; ++j) {
                const double sj = ((dphi[j][0] * og[0] + dphi[j][1] * og[1]) + dphi[j][2] * og[2]) + dphi[j][3] * og[3];
                for (int i = 0; i < NB; ++i) {
                    Kc[i][j] += W * phi[i] * sj;
                    Mc[i][j] += W * phi[i] * phi[j];
                }
            }
        }
        /* physical quadrature points of the inflow faces, and the face matrices */
        double Fc[NB][NB];
        memset(Fc, 0, sizeof(Fc));
        double fx[4][NQ * NQ][3], fl[4][NQ * NQ][4], fw[4][NQ * NQ];
        const int32_t *t = P->tets + 4 * c;
        for (int f = 0; f < 4; ++f) {
            if (!(mask[c] >> f & 1)) continue;
            const double *N = P->normal + 12 * c + 3 * f;
            const double s = (O[0] * N[0] + O[1] * N[1]) + O[2] * N[2];
            int fv[3], m = 0;
            for (int i = 0; i < 4; ++i) if (i != f) fv[m++] = i;
            for (int k = 0; k < NQ * NQ; ++k) {
                double l[4] = {0.0, 0.0, 0.0, 0.0};
                l[fv[0]] = 1.0 - eq[k][0] - eq[k][1];
                l[fv[1]] = eq[k][0];
                l[fv[2]] = eq[k][1];
                for (int d = 0; d < 3; ++d) {
                    fx[f][k][d] = 0.0;
                    for (int i = 0; i < 4; ++i) fx[f][k][d] += l[i] * P->xyz[3 * t[i] + d];
                }
                memcpy(fl[f][k], l, sizeof(l));
                fw[f][k] = fabs(s) * we[k];  /* |Omega.n_f| A_f w_k = |Omega.N_f| w_k */
                double phi[NB];
                basis(l, phi);
                for (int i = 0; i < NB; ++i)
                    for (int j = 0; j < NB; ++j) Fc[i][j] += fw[f][k] * phi[i] * phi[j];
            }
        }
        const int mat = P->material[c];
        for (int g = 0; g < G; ++g) {
            const double sig = P->sigma_t[(size_t)mat * G + g];
            double A[NB][NB], b[NB], x[NB];
            for (int i = 0; i < NB; ++i)
                for (int j = 0; j < NB; ++j) A[i][j] = Kc[i][j] + sig * Mc[i][j] + Fc[i][j];
            const double *qc = q + ((size_t)c * G + g) * NB;
            const double *s1 = P->S1 ? P->S1 + ((size_t)c * G + g) * NB * 3 : NULL;
            for (int i = 0; i < NB; ++i) b[i] = 0.0;
            for (int k = 0; k < NQ * NQ * NQ; ++k) {
                double phi[NB];
                basis(lq[k], phi);
                double src = 0.0;
                for (int m = 0; m < NB; ++m) {
                    src += phi[m] * qc[m];
                    if (s1) src += phi[m] * ((O[0] * s1[3 * m] + O[1] * s1[3 * m + 1]) + O[2] * s1[3 * m + 2]);
                }
                for (int i = 0; i < NB; ++i) b[i] += V * wq[k] * phi[i] * src;
            }
            for (int f = 0; f < 4; ++f) {
                if (!(mask[c] >> f & 1)) continue;
                const int64_t n = P->nbr[4 * c + f];
                for (int k = 0; k < NQ * NQ; ++k) {
                    double up = 0.0, ph[NB];
                    if (n >= 0) {
                        double ln[4];
                        bary(P, n, fx[f][k], ln);
                        basis(ln, ph);
                        const double *pn = psi + ((size_t)n * G + g) * NB;
                        for (int m = 0; m < NB; ++m) up += ph[m] * pn[m];
                    } else if (P->psi_bc) {
                        basis(fl[f][k], ph);
                        const double *pb = P->psi_bc + ((size_t)c * G + g) * NB;
                        for (int m = 0; m < NB; ++m) up += ph[m] * pb[m];
                    }
                    double phi[NB];
                    basis(fl[f][k], phi);
                    for (int i = 0; i < NB; ++i) b[i] += fw[f][k] * phi[i] * up;
                }
            }
            if (lu_solve(A, b, x) != ORA_OK) { status = ORA_ERR_SINGULAR; break; }
            for (int i = 0; i < NB; ++i) psi[((size_t)c * G + g) * NB + i] = x[i];
        }
    }
    free(order);
    return status;
}

/* phi = sum_a w_a psi_a over the listed directions (Eq. 2), nodal [nc][G][10];
 * per-thread partials summed in thread order.  psi_keep: [ndir][nc][G][10] or NULL. */
int ora2_sweep(const ora2_problem *P, const double *q, int ndir, const int32_t *dirs, double *phi, double *psi_keep,
               int nthreads, int *threads)
{
    const size_t n = (size_t)P->nc * P->G * NB;
    memset(phi, 0, sizeof(double) * n);
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
    int nt = nthreads < ndir ? nthreads : ndir;
    if (nt < 1) nt = 1;
#else
    int nt = 1;
#endif
    if (threads) *threads = nt;
    double *part = calloc((size_t)nt * n, sizeof(double));
    if (!part && n > 0) return ORA_ERR_NOMEM;
    int status = ORA_OK;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double *psi = psi_keep ? NULL : malloc(sizeof(double) * (n > 0 ? n : 1));
        double *acc = part + (size_t)tid * n;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < ndir; ++k) {
            int a = dirs[k];
            double *ps = psi_keep ? psi_keep + (size_t)k * n : psi;
            int st = ps ? ora2_sweep_direction(P, a, q, ps) : ORA_ERR_NOMEM;
            if (st != ORA_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                status = st;
                continue;
            }
            const double wa = P->w[a];
            for (size_t i = 0; i < n; ++i) acc[i] += wa * ps[i];
        }
        free(psi);
    }
    for (int t = 0; t < nt; ++t)
        for (size_t i = 0; i < n; ++i) phi[i] += part[(size_t)t * n + i];
    free(part);
    return status;
}
