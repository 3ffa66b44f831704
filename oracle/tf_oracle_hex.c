/*
 * Plain FP64 CPU oracle for the upwind-DG sweep on trilinear hexahedra.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; it shares no code, header or helper with the library.
 * Compiled with -ffp-contract=off.
 *
 * What it computes: the transport problem of Eq. (1) (isotropic scattering)
 * discretised by upwind discontinuous Galerkin on the trilinear hexahedron,
 * the element of the paper's own mini-app meshes (Sec. 2: an orthogonal hex
 * grid twisted along one axis); the per-direction sweep in t-level order
 * (Sec. 2.1, Algorithm 1: all groups inside one element visit); the scalar
 * flux of Eq. (2).
 *
 * Element.  Local vertex v = a + 2b + 4c, (a, b, c) in {0,1}^3, sits at the
 * corner (a, b, c) of the reference cube [0,1]^3.  Basis
 *     b_v(xi) = prod_d (bit d of v ? xi_d : 1 - xi_d),
 * map x(xi) = sum_v x_v b_v(xi), tangents t_k = dx/dxi_k, Jacobian det
 * J = t_0 . (t_1 x t_2).  Face f = 2d + s is the reference face xi_d = s; its
 * face-local nodes k = 0..3 are the vertices whose bit d equals s, in
 * increasing local index.
 *
 * Element integrals (the ingredients of Table 1: f_i f_j det J,
 * f_i df_j/dx det J, face normals, face nodes, element neighbours):
 *     M[i][j]       = int_K b_i b_j dV
 *     Gd[d][i][j]   = int_K b_i (d b_j / d x_d) dV
 *                   = int b_i sum_k cof(J)[d][k] (d b_j / d xi_k) dxi,
 *                     cof(J) = det(J) J^{-T}, column k = t_{k+1} x t_{k+2}
 *     F[f][d][k][l] = int_f N_d b_k b_l,  N = (2s - 1) t_{d+1} x t_{d+2}
 *                     (indices mod 3): the outward area-vector density
 * All integrands are polynomials of degree at most four per reference axis,
 * so the 3-point Gauss-Legendre rule per axis integrates them exactly.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - a face's integrated area vector Nbar_f = int_f N dA is half the cross
 *     product of its diagonals (exact for the bilinear face), computed from
 *     the face's global vertices in a canonical order and then signed
 *     outward, so that two cells sharing a face hold exactly opposite values;
 *   - a face is inflow for Omega iff Omega.Nbar_f < -1e-12 |Nbar_f|, the dot
 *     product evaluated as ((Ox*Nx + Oy*Ny) + Oz*Nz): a twisted (non-planar)
 *     face is wholly inflow or wholly outflow, so the sweep graph stays the
 *     face-adjacency graph oriented by one sign per face;
 *   - the inflow face term uses the signed integrand, -int_f (Omega.N) b_k b_l
 *     (equal to int_f |Omega.N| b_k b_l on a planar face), which keeps the
 *     particle balance exact;
 *   - the upwind trace at a face node is the upwind cell's nodal value at the
 *     same global vertex; boundary inflow is a prescribed isotropic
 *     per-vertex value, or zero (vacuum);
 *   - an element whose Jacobian determinant is not positive at its eight
 *     corners and its 27 quadrature points is rejected.
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
    const int32_t *hexes;     /* [nc][8] */
    const double *mass;       /* [nc][8][8] */
    const double *grad;       /* [nc][3][8][8]  Gd */
    const double *face;       /* [nc][6][3][4][4] F */
    const double *nbar;       /* [nc][6][3] */
    const int32_t *nbr;       /* [nc][6] neighbour across face f, -1 on the boundary */
    const int32_t *nbr_node;  /* [nc][6][4] local index, in the neighbour, of face-local node k (-1 on the boundary) */
    const double *omega;      /* [D][3] */
    const double *w;          /* [D] */
    const uint8_t *inflow;    /* [D][nc] bit f set iff face f is inflow */
    const int32_t *level;     /* [D][nc] */
    const int32_t *material;  /* [nc] */
    const double *sigma_t;    /* [M][G] */
    const double *S1;         /* [nc][G][3] or NULL: extra angular source Omega.S1 (constant per cell) */
    const double *psi_in;     /* [nv][G] or NULL: isotropic inflow on boundary vertices (NULL = vacuum) */
    const uint8_t *lag;       /* [D][nc] or NULL: bit f set iff inflow face f is a lagged back edge */
    const double *psi_prev;   /* [D][nc][G][8] or NULL (zero): the previous transport step's psi, read
                               * on lagged faces */
} orah_problem;

/* face-local node k of face f: the k-th vertex (increasing local index) with bit d equal to s */
static int face_node(int f, int k)
{
    const int d = f / 2, s = f % 2;
    int seen = 0;
    for (int v = 0; v < 8; ++v) {
        if (((v >> d) & 1) != s) continue;
        if (seen == k) return v;
        ++seen;
    }
    return -1;
}

int orah_face_node(int f, int k) { return face_node(f, k); }

/* basis values b[v] and reference derivatives db[v][k] at xi */
static void basis(const double xi[3], double b[8], double db[8][3])
{
    for (int v = 0; v < 8; ++v) {
        double l[3], dl[3];
        for (int d = 0; d < 3; ++d) {
            const int bit = (v >> d) & 1;
            l[d] = bit ? xi[d] : 1.0 - xi[d];
            dl[d] = bit ? 1.0 : -1.0;
        }
        b[v] = l[0] * l[1] * l[2];
        db[v][0] = dl[0] * l[1] * l[2];
        db[v][1] = l[0] * dl[1] * l[2];
        db[v][2] = l[0] * l[1] * dl[2];
    }
}

static void cross(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* tangents t[k][r] = d x_r / d xi_k */
static void tangents(const double X[8][3], const double db[8][3], double t[3][3])
{
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            double s = 0.0;
            for (int v = 0; v < 8; ++v) s += X[v][r] * db[v][k];
            t[k][r] = s;
        }
}

/* 3-point Gauss-Legendre on [0, 1]: nodes 1/2 -+ sqrt(15)/10 and 1/2, weights 5/18, 8/18, 5/18 */
static void gauss3(double x[3], double w[3])
{
    const double h = sqrt(15.0) / 10.0;
    x[0] = 0.5 - h; x[1] = 0.5; x[2] = 0.5 + h;
    w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
}

typedef struct { int32_t v[4]; int64_t cell; int32_t face; } face_rec;

static int face_cmp(const void *pa, const void *pb)
{
    const face_rec *a = pa, *b = pb;
    for (int k = 0; k < 4; ++k)
        if (a->v[k] != b->v[k]) return a->v[k] < b->v[k] ? -1 : 1;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return a->face - b->face;
}

static void sort4(int32_t *v)
{
    for (int i = 1; i < 4; ++i)
        for (int j = i; j > 0 && v[j - 1] > v[j]; --j) { int32_t t = v[j]; v[j] = v[j - 1]; v[j - 1] = t; }
}

/* Element integrals, integrated face area vectors and face neighbours of a hex mesh.
 * Outputs: vol [nc], mass [nc][8][8], grad [nc][3][8][8], face [nc][6][3][4][4],
 * nbar [nc][6][3], nbr [nc][6], nbr_node [nc][6][4].  ORA_ERR_MESH for a vertex
 * index out of range, a non-positive Jacobian at a corner or quadrature point,
 * or a face shared by more than two cells. */
int orah_geometry(int64_t nv, const double *xyz, int64_t nc, const int32_t *hexes, double *vol,
                  double *mass, double *grad, double *face, double *nbar, int32_t *nbr, int32_t *nbr_node)
{
    double gx[3], gw[3];
    gauss3(gx, gw);
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t *hx = hexes + 8 * c;
        double X[8][3];
        for (int v = 0; v < 8; ++v) {
            if (hx[v] < 0 || hx[v] >= nv) return ORA_ERR_MESH;
            for (int r = 0; r < 3; ++r) X[v][r] = xyz[3 * hx[v] + r];
        }
        double b[8], db[8][3], t[3][3], cof[3][3];
        /* corners */
        for (int v = 0; v < 8; ++v) {
            double xi[3] = {(double)(v & 1), (double)((v >> 1) & 1), (double)((v >> 2) & 1)};
            basis(xi, b, db);
            tangents(X, db, t);
            cross(t[1], t[2], cof[0]);
            double det = t[0][0] * cof[0][0] + t[0][1] * cof[0][1] + t[0][2] * cof[0][2];
            if (!(det > 0.0)) return ORA_ERR_MESH;
        }
        double *Mc = mass + 64 * c, *Gc = grad + 192 * c, *Fc = face + 288 * c;
        memset(Mc, 0, 64 * sizeof(double));
        memset(Gc, 0, 192 * sizeof(double));
        memset(Fc, 0, 288 * sizeof(double));
        double V = 0.0;
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
                for (int r = 0; r < 3; ++r) {
                    double xi[3] = {gx[p], gx[q], gx[r]};
                    const double wt = gw[p] * gw[q] * gw[r];
                    basis(xi, b, db);
                    tangents(X, db, t);
                    /* cof[k] = column k of cof(J) = t_{k+1} x t_{k+2} */
                    for (int k = 0; k < 3; ++k) cross(t[(k + 1) % 3], t[(k + 2) % 3], cof[k]);
                    double det = t[0][0] * cof[0][0] + t[0][1] * cof[0][1] + t[0][2] * cof[0][2];
                    if (!(det > 0.0)) return ORA_ERR_MESH;
                    V += wt * det;
                    for (int i = 0; i < 8; ++i)
                        for (int j = 0; j < 8; ++j) Mc[8 * i + j] += wt * det * b[i] * b[j];
                    for (int d = 0; d < 3; ++d)
                        for (int j = 0; j < 8; ++j) {
                            /* (d b_j / d x_d) det J */
                            double gj = cof[0][d] * db[j][0] + cof[1][d] * db[j][1] + cof[2][d] * db[j][2];
                            for (int i = 0; i < 8; ++i) Gc[64 * d + 8 * i + j] += wt * b[i] * gj;
                        }
                }
        vol[c] = V;
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2, s = f % 2, e1 = (d + 1) % 3, e2 = (d + 2) % 3;
            int node[4];
            for (int k = 0; k < 4; ++k) node[k] = face_node(f, k);
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    double xi[3];
                    xi[d] = (double)s;
                    xi[e1] = gx[p];
                    xi[e2] = gx[q];
                    const double wt = gw[p] * gw[q];
                    basis(xi, b, db);
                    tangents(X, db, t);
                    double N[3];
                    cross(t[e1], t[e2], N);
                    if (!s) { N[0] = -N[0]; N[1] = -N[1]; N[2] = -N[2]; }
                    for (int dd = 0; dd < 3; ++dd)
                        for (int k = 0; k < 4; ++k)
                            for (int l = 0; l < 4; ++l)
                                Fc[48 * f + 16 * dd + 4 * k + l] += wt * N[dd] * b[node[k]] * b[node[l]];
                }
            /* integrated area vector from the diagonals, canonical order: each diagonal runs
             * from its smaller global vertex id to its larger; the diagonal holding the
             * smallest id comes first */
            int32_t g0 = hx[node[0]], g1 = hx[node[1]], g2 = hx[node[2]], g3 = hx[node[3]];
            int32_t a0 = g0 < g3 ? g0 : g3, a1 = g0 < g3 ? g3 : g0;
            int32_t b0 = g1 < g2 ? g1 : g2, b1 = g1 < g2 ? g2 : g1;
            if (b0 < a0) { int32_t u = a0; a0 = b0; b0 = u; u = a1; a1 = b1; b1 = u; }
            double dA[3], dB[3], Nb[3];
            for (int r = 0; r < 3; ++r) {
                dA[r] = xyz[3 * a1 + r] - xyz[3 * a0 + r];
                dB[r] = xyz[3 * b1 + r] - xyz[3 * b0 + r];
            }
            cross(dA, dB, Nb);
            double own = 0.0; /* the quadrature's integrated normal, only for the orientation */
            for (int dd = 0; dd < 3; ++dd) {
                double sd = 0.0;
                for (int k = 0; k < 16; ++k) sd += Fc[48 * f + 16 * dd + k];
                own += sd * Nb[dd];
            }
            const double sg = own < 0.0 ? -0.5 : 0.5;
            for (int r = 0; r < 3; ++r) nbar[18 * c + 3 * f + r] = sg * Nb[r];
        }
    }
    /* face matching by sorting (sorted vertex quadruple, cell, face) records */
    face_rec *rec = malloc(sizeof(face_rec) * (size_t)(6 * nc > 0 ? 6 * nc : 1));
    if (!rec) return ORA_ERR_NOMEM;
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 6; ++f) {
            face_rec *r = rec + 6 * c + f;
            for (int k = 0; k < 4; ++k) r->v[k] = hexes[8 * c + face_node(f, k)];
            sort4(r->v);
            r->cell = c;
            r->face = f;
        }
    qsort(rec, (size_t)(6 * nc), sizeof(face_rec), face_cmp);
    for (int64_t i = 0; i < 6 * nc; ++i) nbr[i] = -1;
    for (int64_t i = 0; i < 24 * nc; ++i) nbr_node[i] = -1;
    int64_t i = 0;
    while (i < 6 * nc) {
        int64_t j = i + 1;
        while (j < 6 * nc && memcmp(rec[j].v, rec[i].v, sizeof(rec[i].v)) == 0) ++j;
        if (j - i > 2) { free(rec); return ORA_ERR_MESH; }
        if (j - i == 2) {
            for (int s = 0; s < 2; ++s) {
                int64_t c = rec[i + s].cell, n = rec[i + 1 - s].cell;
                int f = rec[i + s].face;
                nbr[6 * c + f] = (int32_t)n;
                for (int k = 0; k < 4; ++k) {
                    int32_t gv = hexes[8 * c + face_node(f, k)];
                    for (int v = 0; v < 8; ++v)
                        if (hexes[8 * n + v] == gv) nbr_node[24 * c + 4 * f + k] = v;
                }
            }
        }
        i = j;
    }
    free(rec);
    return ORA_OK;
}

/* Face classification and t-levels per direction (Sec. 2.1), Kahn's algorithm as
 * for the tetrahedral oracle, over six faces.  ORA_ERR_CYCLE if a cell is never reached.
 *
 * With lag != NULL ([D][nc]) cycles are broken instead (the paper assumes an acyclic
 * graph; lagging is the usual remedy, not the paper's).  Whenever no cell is ready, a
 * walk starts at the lowest-numbered waiting cell and steps to the upwind neighbour
 * across its lowest-numbered open face (inflow, interior, not reached, not lagged);
 * every waiting cell has one, so the walk comes back to a cell it has visited, and the
 * face it would cross then closes a cycle: that one face is lagged (it will read the
 * upwind cell's psi of the previous transport step) and the ordering continues.
 * Lagged faces do not count for the t-levels. */
int orah_graph_lag(int64_t nc, const int32_t *nbr, const double *nbar, int D, const double *omega,
                   uint8_t *inflow, int32_t *level, uint8_t *lag)
{
    int32_t *indeg = malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t *queue = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t *walk = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    uint8_t *reached = malloc((size_t)(nc > 0 ? nc : 1));
    if (!indeg || !queue || !walk || !reached) {
        free(indeg); free(queue); free(walk); free(reached);
        return ORA_ERR_NOMEM;
    }
    int status = ORA_OK;
    for (int a = 0; a < D && status == ORA_OK; ++a) {
        const double *O = omega + 3 * a;
        uint8_t *mask = inflow + (size_t)a * nc;
        int32_t *lev = level + (size_t)a * nc;
        uint8_t *lg = lag ? lag + (size_t)a * nc : NULL;
        for (int64_t c = 0; c < nc; ++c) {
            uint8_t m = 0;
            for (int f = 0; f < 6; ++f) {
                const double *N = nbar + 18 * c + 3 * f;
                double s = (O[0] * N[0] + O[1] * N[1]) + O[2] * N[2];
                double eps = 1e-12 * sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
                if (s < -eps) m |= (uint8_t)(1u << f);
            }
            mask[c] = m;
            if (lg) lg[c] = 0;
        }
        int64_t head = 0, tail = 0, next = 0;
        for (int64_t c = 0; c < nc; ++c) {
            int deg = 0;
            for (int f = 0; f < 6; ++f)
                if ((mask[c] >> f & 1) && nbr[6 * c + f] >= 0) ++deg;
            indeg[c] = deg;
            lev[c] = 0;
            walk[c] = -1;
            reached[c] = deg == 0;
            if (deg == 0) queue[tail++] = c;
        }
        int64_t stamp = 0;
        for (;;) {
            while (head < tail) {
                int64_t c = queue[head++];
                for (int f = 0; f < 6; ++f) {
                    int64_t n = nbr[6 * c + f];
                    if (n < 0 || reached[n]) continue;
                    int down = 0;
                    for (int g = 0; g < 6; ++g)
                        if (nbr[6 * n + g] == c && (mask[n] >> g & 1) && !(lg && (lg[n] >> g & 1))) down = 1;
                    if (!down) continue;
                    if (lev[n] < lev[c] + 1) lev[n] = lev[c] + 1;
                    if (--indeg[n] == 0) {
                        reached[n] = 1;
                        queue[tail++] = n;
                    }
                }
            }
            if (tail == nc || !lg) break;
            /* no cell is ready: walk upwind from the lowest-numbered waiting cell to a cycle */
            while (reached[next]) ++next;
            int64_t cur = next;
            walk[cur] = stamp;
            for (;;) {
                int fo = -1;
                int64_t n = -1;
                for (int f = 0; f < 6 && fo < 0; ++f) {
                    n = nbr[6 * cur + f];
                    if ((mask[cur] >> f & 1) && !(lg[cur] >> f & 1) && n >= 0 && !reached[n]) fo = f;
                }
                if (fo < 0) { status = ORA_ERR_CYCLE; break; }  /* cannot happen: cur waits on someone */
                if (walk[n] == stamp) {  /* cur -> n closes a cycle: lag that face */
                    lg[cur] |= (uint8_t)(1u << fo);
                    if (--indeg[cur] == 0) {
                        reached[cur] = 1;
                        queue[tail++] = cur;
                    }
                    break;
                }
                walk[n] = stamp;
                cur = n;
            }
            ++stamp;
            if (status != ORA_OK) break;
        }
        if (tail != nc && status == ORA_OK) status = ORA_ERR_CYCLE;
    }
    free(indeg);
    free(queue);
    free(walk);
    free(reached);
    return status;
}

int orah_graph(int64_t nc, const int32_t *nbr, const double *nbar, int D, const double *omega,
               uint8_t *inflow, int32_t *level)
{
    return orah_graph_lag(nc, nbr, nbar, D, omega, inflow, level, NULL);
}

/* Gaussian elimination with partial pivoting on an 8x8 system. */
static int lu_solve8(double A[8][8], double b[8], double x[8])
{
    for (int k = 0; k < 8; ++k) {
        int p = k;
        for (int i = k + 1; i < 8; ++i)
            if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
        if (A[p][k] == 0.0) return ORA_ERR_SINGULAR;
        if (p != k) {
            for (int j = 0; j < 8; ++j) { double u = A[k][j]; A[k][j] = A[p][j]; A[p][j] = u; }
            double u = b[k]; b[k] = b[p]; b[p] = u;
        }
        for (int i = k + 1; i < 8; ++i) {
            double m = A[i][k] / A[k][k];
            for (int j = k; j < 8; ++j) A[i][j] -= m * A[k][j];
            b[i] -= m * b[k];
        }
    }
    for (int i = 7; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < 8; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return ORA_OK;
}

/* Sweep one direction for all groups.  For every cell in increasing (t-level,
 * cell id) order and every group g, solve the upwind-DG local system (weak form
 * of Eq. (1) integrated back by parts, upwind trace on the inflow faces):
 *
 *   sum_j [ sum_d Omega_d Gd[d][i][j] + sum_{f inflow} Fin_f[i][j] + sigma_t,g M[i][j] ] psi_j
 *     = sum_j M[i][j] q_j + (Omega.S1_g) sum_j M[i][j] + sum_{f inflow} sum_j Fin_f[i][j] psi_up,j
 *
 * with Fin_f[k][l] = -sum_d Omega_d F[f][d][k][l] on face f's nodes (zero elsewhere).
 * q is the isotropic angular source per steradian, nodal [nc][G][8]; psi is [nc][G][8]. */
int orah_sweep_direction(const orah_problem *P, int a, const double *q, double *psi)
{
    const int64_t nc = P->nc;
    const int G = P->G;
    const uint8_t *mask = P->inflow + (size_t)a * nc;
    const int32_t *lev = P->level + (size_t)a * nc;
    const double *O = P->omega + 3 * a;
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
        const double *Mc = P->mass + 64 * c, *Gc = P->grad + 192 * c, *Fc = P->face + 288 * c;
        double S[8][8]; /* sum_d Omega_d Gd[d] */
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                S[i][j] = (O[0] * Gc[8 * i + j] + O[1] * Gc[64 + 8 * i + j]) + O[2] * Gc[128 + 8 * i + j];
        double Fin[6][4][4];
        for (int f = 0; f < 6; ++f)
            for (int k = 0; k < 4; ++k)
                for (int l = 0; l < 4; ++l) {
                    const double *F = Fc + 48 * f + 4 * k + l;
                    Fin[f][k][l] = -((O[0] * F[0] + O[1] * F[16]) + O[2] * F[32]);
                }
        double rowm[8];
        for (int i = 0; i < 8; ++i) {
            rowm[i] = 0.0;
            for (int j = 0; j < 8; ++j) rowm[i] += Mc[8 * i + j];
        }
        const int m = P->material[c];
        for (int g = 0; g < G; ++g) {
            const double sig = P->sigma_t[(size_t)m * G + g];
            double A[8][8], b[8], x[8];
            const double *qc = q + ((size_t)c * G + g) * 8;
            for (int i = 0; i < 8; ++i) {
                b[i] = 0.0;
                for (int j = 0; j < 8; ++j) {
                    A[i][j] = S[i][j] + sig * Mc[8 * i + j];
                    b[i] += Mc[8 * i + j] * qc[j];
                }
            }
            if (P->S1) {
                const double *s1 = P->S1 + ((size_t)c * G + g) * 3;
                double os = O[0] * s1[0] + O[1] * s1[1] + O[2] * s1[2];
                for (int i = 0; i < 8; ++i) b[i] += os * rowm[i];
            }
            for (int f = 0; f < 6; ++f) {
                if (!(mask[c] >> f & 1)) continue;
                const int64_t n = P->nbr[6 * c + f];
                const int lagged = P->lag && (P->lag[(size_t)a * nc + c] >> f & 1);
                double up[4];
                for (int k = 0; k < 4; ++k) {
                    const int v = face_node(f, k);
                    if (n >= 0 && lagged)  /* back edge: the upwind cell's psi of the previous step */
                        up[k] = P->psi_prev ? P->psi_prev[(((size_t)a * nc + n) * G + g) * 8 + P->nbr_node[24 * c + 4 * f + k]]
                                            : 0.0;
                    else if (n >= 0)
                        up[k] = psi[((size_t)n * G + g) * 8 + P->nbr_node[24 * c + 4 * f + k]];
                    else if (P->psi_in)
                        up[k] = P->psi_in[(size_t)P->hexes[8 * c + v] * G + g];
                    else
                        up[k] = 0.0;
                }
                for (int k = 0; k < 4; ++k) {
                    const int i = face_node(f, k);
                    for (int l = 0; l < 4; ++l) {
                        A[i][face_node(f, l)] += Fin[f][k][l];
                        b[i] += Fin[f][k][l] * up[l];
                    }
                }
            }
            if (lu_solve8(A, b, x) != ORA_OK) { status = ORA_ERR_SINGULAR; break; }
            for (int i = 0; i < 8; ++i) psi[((size_t)c * G + g) * 8 + i] = x[i];
        }
    }
    free(order);
    return status;
}

/* Sweep the listed directions and accumulate phi = sum_a w_a psi_a (Eq. 2), nodal
 * [nc][G][8]; directions spread over OpenMP threads with per-thread partial sums
 * added in thread order.  psi_keep (or NULL) receives [ndir][nc][G][8]. */
int orah_sweep(const orah_problem *P, const double *q, int ndir, const int32_t *dirs,
               double *phi, double *psi_keep, int nthreads, int *threads)
{
    const size_t n = (size_t)P->nc * P->G * 8;
    memset(phi, 0, sizeof(double) * n);
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
    int nt = nthreads < ndir ? nthreads : ndir;
    if (nt < 1) nt = 1;
#else
    int nt = 1;
#endif
    if (threads) *threads = nt;
    double *part = calloc((size_t)nt * (n > 0 ? n : 1), sizeof(double));
    if (!part) return ORA_ERR_NOMEM;
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
            int st = ps ? orah_sweep_direction(P, a, q, ps) : ORA_ERR_NOMEM;
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
