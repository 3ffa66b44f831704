/*
 * Plain FP64 CPU oracle for the unstructured S_N transport sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: it exists so that tests, the smoke check and the bench's
 * CPU-baseline leg can compare the CUDA library against an obviously correct
 * reference.  It shares no code, header or helper with the library.
 *
 * Every quantity is FP64; the file is compiled with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * What it computes (paper: Elwood et al., "An Asynchronous Many-Task
 * Algorithm for Unstructured S_N Transport on Shared Memory Systems"):
 *   - the steady multigroup transport problem of Eq. (1) with isotropic
 *     scattering, discretised by upwind discontinuous Galerkin on linear
 *     tetrahedra (the element-matrix ingredients of Table 1:
 *     f_i df_j/dx det J, f_i f_j det J, face normals, face nodes, element
 *     neighbours), S_N directions from a product quadrature, energy groups;
 *   - the per-direction sweep in dependency (t-level) order, Sec. 2.1 and
 *     Algorithm 1 (every group solved inside one element visit);
 *   - the scalar flux by quadrature, Eq. (2).
 * The source update, stopping test and integrated flux (Eq. 3) are plain
 * numpy in oracle/__init__.py.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - face f of a tetrahedron is the face opposite local vertex f;
 *   - face normals are area-weighted and computed from the face's global
 *     vertices in increasing id order, then flipped to point outward, so the
 *     two cells sharing a face hold exactly opposite normals;
 *   - a face is inflow for direction Omega iff Omega.N < -1e-12 |N|, with the
 *     dot product evaluated as ((Ox*Nx + Oy*Ny) + Oz*Nz);
 *   - the upwind trace at a face vertex is the upwind cell's nodal value at
 *     the same global vertex; boundary inflow is a prescribed isotropic
 *     per-vertex value, or zero (vacuum);
 *   - t-levels: 0 with no interior inflow face, else 1 + max over upwinds;
 *     a dependency cycle is an error.
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
#define ORA_ERR_MESH 2
#define ORA_ERR_CYCLE 3
#define ORA_ERR_NOMEM 5
#define ORA_ERR_SINGULAR 9

typedef struct {
    int64_t nc;               /* cells */
    int64_t nv;               /* vertices */
    int32_t G;                /* groups */
    int32_t D;                /* directions */
    const double *xyz;        /* [nv][3] */
    const int32_t *tets;      /* [nc][4] */
    const double *vol;        /* [nc] */
    const double *grad;       /* [nc][4][3]  gradient of basis b_j */
    const double *normal;     /* [nc][4][3]  area-weighted outward normal of face f */
    const int32_t *nbr;       /* [nc][4]     neighbour across face f, -1 on the boundary */
    const int32_t *nbr_node;  /* [nc][4][4]  [c][f][i]: local index, in the neighbour across f, of local vertex i of c (-1 for i == f or no neighbour) */
    const double *omega;      /* [D][3] */
    const double *w;          /* [D] */
    const uint8_t *inflow;    /* [D][nc]     bit f set iff face f is inflow */
    const int32_t *level;     /* [D][nc] */
    const int32_t *material;  /* [nc] */
    const double *sigma_t;    /* [M][G] */
    const double *S1;         /* [nc][G][3] or NULL: extra angular source Omega.S1 (constant per cell) */
    const double *psi_in;     /* [nv][G] or NULL: isotropic inflow on boundary vertices (NULL = vacuum) */
} ora_problem;

/* ------------------------------------------------------------ quadrature */

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton's method on
 * P_n, evaluated with the three-term recurrence (k+1)P_{k+1} = (2k+1)x P_k - k P_{k-1}. */
int ora_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return ORA_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        /* i-th largest root; stored at position n-1-i so the output ascends */
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z = z - dz;
            if (fabs(dz) <= 1e-16) break;
        }
        /* derivative at the final node */
        double p0 = 1.0, p1 = z;
        for (int k = 1; k < n; ++k) {
            double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return ORA_OK;
}

/* Product quadrature: n_polar Gauss-Legendre cosines mu_i times n_az azimuths
 * phi_k = (k + 1/2) 2 pi / n_az.  Direction a = i * n_az + k,
 * Omega = (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu), weight w_i 2 pi / n_az,
 * so the weights sum to 4 pi. */
int ora_product_quadrature(int n_polar, int n_az, double *omega, double *w)
{
    if (n_polar < 1 || n_az < 1) return ORA_ERR_ARG;
    double *mu = malloc(sizeof(double) * n_polar), *wm = malloc(sizeof(double) * n_polar);
    if (!mu || !wm) { free(mu); free(wm); return ORA_ERR_NOMEM; }
    ora_gauss_legendre(n_polar, mu, wm);
    for (int i = 0; i < n_polar; ++i) {
        double s = sqrt(1.0 - mu[i] * mu[i]);
        for (int k = 0; k < n_az; ++k) {
            double ph = (k + 0.5) * (2.0 * M_PI / n_az);
            int a = i * n_az + k;
            omega[3 * a + 0] = s * cos(ph);
            omega[3 * a + 1] = s * sin(ph);
            omega[3 * a + 2] = mu[i];
            w[a] = wm[i] * (2.0 * M_PI / n_az);
        }
    }
    free(mu);
    free(wm);
    return ORA_OK;
}

/* ------------------------------------------------------------ geometry */

typedef struct { int32_t v[3]; int64_t cell; int32_t face; } face_rec;

static int face_cmp(const void *pa, const void *pb)
{
    const face_rec *a = pa, *b = pb;
    for (int k = 0; k < 3; ++k) {
        if (a->v[k] != b->v[k]) return a->v[k] < b->v[k] ? -1 : 1;
    }
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return a->face - b->face;
}

static void sort3(int32_t *v)
{
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

/* Volumes, basis gradients, area-weighted outward face normals and the face
 * neighbour maps of a tetrahedral mesh.  Returns ORA_ERR_MESH for a tetrahedron
 * with non-positive volume, a vertex index out of range, or a face shared by
 * more than two cells. */
int ora_geometry(int64_t nv, const double *xyz, int64_t nc, const int32_t *tets,
                 double *vol, double *grad, double *normal, int32_t *nbr, int32_t *nbr_node)
{
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t *t = tets + 4 * c;
        for (int i = 0; i < 4; ++i)
            if (t[i] < 0 || t[i] >= nv) return ORA_ERR_MESH;
        const double *x0 = xyz + 3 * t[0];
        double J[3][3]; /* J[r][k] = x_{k+1}[r] - x_0[r]  (columns are edges) */
        for (int k = 0; k < 3; ++k)
            for (int r = 0; r < 3; ++r) J[r][k] = xyz[3 * t[k + 1] + r] - x0[r];
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                   - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                   + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0)) return ORA_ERR_MESH;
        vol[c] = det / 6.0;
        /* inverse of J by cofactors; row k of J^{-1} is the gradient of b_{k+1} */
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        double *gc = grad + 12 * c;
        for (int d = 0; d < 3; ++d) {
            gc[3 * 1 + d] = inv[0][d];
            gc[3 * 2 + d] = inv[1][d];
            gc[3 * 3 + d] = inv[2][d];
            gc[3 * 0 + d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
        }
        for (int f = 0; f < 4; ++f) {
            int32_t s[3];
            int k = 0;
            for (int i = 0; i < 4; ++i)
                if (i != f) s[k++] = t[i];
            sort3(s);
            const double *xa = xyz + 3 * s[0], *xb = xyz + 3 * s[1], *xc = xyz + 3 * s[2];
            double e1[3], e2[3], N[3];
            for (int d = 0; d < 3; ++d) { e1[d] = xb[d] - xa[d]; e2[d] = xc[d] - xa[d]; }
            N[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
            N[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
            N[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
            const double *xo = xyz + 3 * t[f];
            double side = (N[0] * (xo[0] - xa[0]) + N[1] * (xo[1] - xa[1])) + N[2] * (xo[2] - xa[2]);
            if (side > 0.0) { N[0] = -N[0]; N[1] = -N[1]; N[2] = -N[2]; }
            for (int d = 0; d < 3; ++d) normal[12 * c + 3 * f + d] = N[d];
        }
    }
    /* face matching by sorting all (sorted vertex triple, cell, face) records */
    face_rec *rec = malloc(sizeof(face_rec) * (size_t)(4 * nc));
    if (!rec && nc > 0) return ORA_ERR_NOMEM;
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 4; ++f) {
            face_rec *r = rec + 4 * c + f;
            int k = 0;
            for (int i = 0; i < 4; ++i)
                if (i != f) r->v[k++] = tets[4 * c + i];
            sort3(r->v);
            r->cell = c;
            r->face = f;
        }
    qsort(rec, (size_t)(4 * nc), sizeof(face_rec), face_cmp);
    for (int64_t i = 0; i < 4 * nc; ++i) nbr[i] = -1;
    for (int64_t i = 0; i < 16 * nc; ++i) nbr_node[i] = -1;
    int64_t i = 0;
    while (i < 4 * nc) {
        int64_t j = i + 1;
        while (j < 4 * nc && memcmp(rec[j].v, rec[i].v, sizeof(rec[i].v)) == 0) ++j;
        if (j - i > 2) { free(rec); return ORA_ERR_MESH; }
        if (j - i == 2) {
            for (int s = 0; s < 2; ++s) {
                int64_t c = rec[i + s].cell, n = rec[i + 1 - s].cell;
                int f = rec[i + s].face;
                nbr[4 * c + f] = (int32_t)n;
                for (int a = 0; a < 4; ++a) {
                    if (a == f) continue;
                    for (int b = 0; b < 4; ++b)
                        if (tets[4 * n + b] == tets[4 * c + a]) nbr_node[16 * c + 4 * f + a] = b;
                }
            }
        }
        i = j;
    }
    free(rec);
    return ORA_OK;
}

/* ------------------------------------------------------------ graph */

/* Face classification and t-levels for each direction (Sec. 2.1: the sweep
 * dependencies form a DAG; buckets hold the cells of one t-level).
 * Kahn's algorithm: cells with no interior inflow face start at level 0; a
 * cell's level is one more than the largest level among its upwind cells.
 * Cells never reached mean a cycle: ORA_ERR_CYCLE. */
int ora_graph(int64_t nc, const int32_t *nbr, const double *normal, int D, const double *omega,
              uint8_t *inflow, int32_t *level)
{
    int32_t *indeg = malloc(sizeof(int32_t) * (size_t)nc);
    int64_t *queue = malloc(sizeof(int64_t) * (size_t)nc);
    if ((!indeg || !queue) && nc > 0) { free(indeg); free(queue); return ORA_ERR_NOMEM; }
    int status = ORA_OK;
    for (int a = 0; a < D && status == ORA_OK; ++a) {
        const double *O = omega + 3 * a;
        uint8_t *mask = inflow + (size_t)a * nc;
        int32_t *lev = level + (size_t)a * nc;
        for (int64_t c = 0; c < nc; ++c) {
            uint8_t m = 0;
            for (int f = 0; f < 4; ++f) {
                const double *N = normal + 12 * c + 3 * f;
                double s = (O[0] * N[0] + O[1] * N[1]) + O[2] * N[2];
                double eps = 1e-12 * sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
                if (s < -eps) m |= (uint8_t)(1u << f);
            }
            mask[c] = m;
        }
        int64_t head = 0, tail = 0;
        for (int64_t c = 0; c < nc; ++c) {
            int deg = 0;
            for (int f = 0; f < 4; ++f)
                if ((mask[c] >> f & 1) && nbr[4 * c + f] >= 0) ++deg;
            indeg[c] = deg;
            lev[c] = 0;
            if (deg == 0) queue[tail++] = c;
        }
        while (head < tail) {
            int64_t c = queue[head++];
            for (int f = 0; f < 4; ++f) {
                int64_t n = nbr[4 * c + f];
                if (n < 0) continue;
                /* is c upwind of n?  n has an inflow face whose neighbour is c */
                int down = 0;
                for (int g = 0; g < 4; ++g)
                    if (nbr[4 * n + g] == c && (mask[n] >> g & 1)) down = 1;
                if (!down) continue;
                if (lev[n] < lev[c] + 1) lev[n] = lev[c] + 1;
                if (--indeg[n] == 0) queue[tail++] = n;
            }
        }
        if (tail != nc) status = ORA_ERR_CYCLE;
    }
    free(indeg);
    free(queue);
    return status;
}

/* ------------------------------------------------------------ local solve */

/* Gaussian elimination with partial pivoting on a 4x4 system. */
static int lu_solve4(double A[4][4], double b[4], double x[4])
{
    for (int k = 0; k < 4; ++k) {
        int p = k;
        for (int i = k + 1; i < 4; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == 0.0) return ORA_ERR_SINGULAR;
        if (p != k) {
            for (int j = 0; j < 4; ++j) { double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < 4; ++i) {
            double m = A[i][k] / A[k][k];
            for (int j = k; j < 4; ++j) A[i][j] -= m * A[k][j];
            b[i] -= m * b[k];
        }
    }
    for (int i = 3; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < 4; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return ORA_OK;
}

/* Sweep one direction for all groups.
 *
 * For every cell, in increasing (t-level, cell id) order, and every group g,
 * solve the upwind-DG local system (weak form of Eq. (1), integrated back by
 * parts, upwind trace on inflow faces):
 *
 *   sum_j [ int_K b_i Omega.grad b_j  +  sum_{f inflow} |Omega.n_f| int_f b_i b_j
 *           + sigma_t,g int_K b_i b_j ] psi_j
 *     = int_K b_i q_g  +  int_K b_i (Omega.S1_g)  +  sum_{f inflow} |Omega.n_f| int_f b_i psi_up
 *
 * with int_K b_i d_x b_j = (V/4) d_x b_j, int_K b_i b_j = (V/20)(1 + delta_ij),
 * int_f b_i b_j = (A_f/12)(1 + delta_ij) for i, j on face f, |Omega.n_f| A_f = |Omega.N_f|.
 * q is the isotropic angular source per steradian, nodal [nc][G][4].
 * psi_out is [nc][G][4]. */
int ora_sweep_direction(const ora_problem *P, int a, const double *q, double *psi)
{
    const int64_t nc = P->nc;
    const int G = P->G;
    const uint8_t *mask = P->inflow + (size_t)a * nc;
    const int32_t *lev = P->level + (size_t)a * nc;
    const double *O = P->omega + 3 * a;
    /* counting sort of cells by level (stable, so ties stay in id order) */
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
        double stream[4]; /* (V/4) Omega.grad b_j */
        for (int j = 0; j < 4; ++j)
            stream[j] = (V / 4.0) * (O[0] * gr[3 * j] + O[1] * gr[3 * j + 1] + O[2] * gr[3 * j + 2]);
        double sabs[4];
        for (int f = 0; f < 4; ++f) {
            const double *N = P->normal + 12 * c + 3 * f;
            sabs[f] = fabs(O[0] * N[0] + O[1] * N[1] + O[2] * N[2]);
        }
        const int m = P->material[c];
        for (int g = 0; g < G; ++g) {
            const double sig = P->sigma_t[(size_t)m * G + g];
            double A[4][4], b[4], x[4];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    A[i][j] = stream[j] + sig * (V / 20.0) * (i == j ? 2.0 : 1.0);
            const double *qc = q + ((size_t)c * G + g) * 4;
            for (int i = 0; i < 4; ++i) {
                b[i] = 0.0;
                for (int j = 0; j < 4; ++j) b[i] += (V / 20.0) * (i == j ? 2.0 : 1.0) * qc[j];
            }
            if (P->S1) {
                const double *s1 = P->S1 + ((size_t)c * G + g) * 3;
                double os = O[0] * s1[0] + O[1] * s1[1] + O[2] * s1[2];
                for (int i = 0; i < 4; ++i) b[i] += (V / 4.0) * os;
            }
            for (int f = 0; f < 4; ++f) {
                if (!(mask[c] >> f & 1)) continue;
                const double t = sabs[f] / 12.0;
                double up[4] = {0.0, 0.0, 0.0, 0.0}; /* upwind trace at local vertex i of c */
                const int64_t n = P->nbr[4 * c + f];
                for (int i = 0; i < 4; ++i) {
                    if (i == f) continue;
                    if (n >= 0) {
                        int k = P->nbr_node[16 * c + 4 * f + i];
                        up[i] = psi[((size_t)n * G + g) * 4 + k];
                    } else if (P->psi_in) {
                        up[i] = P->psi_in[(size_t)P->tets[4 * c + i] * G + g];
                    }
                }
                for (int i = 0; i < 4; ++i) {
                    if (i == f) continue;
                    for (int j = 0; j < 4; ++j) {
                        if (j == f) continue;
                        double mf = t * (i == j ? 2.0 : 1.0);
                        A[i][j] += mf;
                        b[i] += mf * up[j];
                    }
                }
            }
            if (lu_solve4(A, b, x) != ORA_OK) { status = ORA_ERR_SINGULAR; break; }
            for (int i = 0; i < 4; ++i) psi[((size_t)c * G + g) * 4 + i] = x[i];
        }
    }
    free(order);
    return status;
}

/* Sweep the listed directions and accumulate phi = sum_a w_a psi_a (Eq. 2),
 * nodal [nc][G][4].  With OpenMP, directions are spread over threads, each
 * with its own partial phi, summed in thread order at the end.
 * If psi_keep is not NULL it receives psi of the listed directions,
 * [ndir][nc][G][4].  Returns the number of threads used through *threads. */
int ora_sweep(const ora_problem *P, const double *q, int ndir, const int32_t *dirs,
              double *phi, double *psi_keep, int nthreads, int *threads)
{
    const size_t n = (size_t)P->nc * P->G * 4;
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
            int st = ps ? ora_sweep_direction(P, a, q, ps) : ORA_ERR_NOMEM;
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
