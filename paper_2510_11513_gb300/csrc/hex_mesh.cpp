// Host geometry of a mesh of trilinear hexahedra (FP64, no floating-point contraction).
//
// Element: local vertex v = a + 2b + 4c sits at the corner (a, b, c) of the reference
// cube [0,1]^3; basis b_v(xi) = prod_d (bit d of v ? xi_d : 1 - xi_d); map
// x(xi) = sum_v x_v b_v(xi).  Face f = 2d + s is the reference face xi_d = s, its
// face-local nodes the four vertices with bit d equal to s in increasing local index.
//
// The element integrals of Table 1 (f_i f_j det J, f_i df_j/dx det J, face
// normals) are computed by exact polynomial algebra instead of quadrature: the map is
// trilinear, so the tangents t_k = dx/dxi_k, the cofactor columns t_{k+1} x t_{k+2}
// (the columns of det J times J^{-T}) and det J are polynomials of degree at most two per
// reference axis; each integrand is such a polynomial times basis
// functions, integrated monomial by monomial with
//     int_0^1 xi^m dxi = 1/(m+1),  int xi^m (1-xi) = 1/((m+1)(m+2)), ...
//
// Outputs per cell: mass M[i][j] = int b_i b_j; streaming G[d][i][j] = int b_i d b_j/dx_d;
// face F[f][d][k][l] = int_f N_d b_k b_l with N the outward area-vector density; the
// integrated face area vector Nbar_f (half the cross product of the face diagonals, in a
// canonical order of the face's global vertices, signed outward), which classifies the
// face for a direction exactly as for the tetrahedra (inflow iff Omega.Nbar_f < -1e-12
// |Nbar_f|), so that the two cells sharing a face hold exactly opposite vectors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "tf_internal.h"

namespace tf {

namespace {

constexpr int PD = 5;  // exponents 0..4 per axis

struct Poly {
    int deg[3] = {0, 0, 0};  // highest exponent per axis that may be non-zero
    double c[PD][PD][PD];    // c[e0][e1][e2]: coefficient of xi0^e0 xi1^e1 xi2^e2
    Poly() { std::memset(c, 0, sizeof(c)); }
};

inline int bit(int v, int d) { return (v >> d) & 1; }

// sum_v val[v] b_v as a polynomial
Poly trilinear(const double val[8])
{
    Poly p;
    p.deg[0] = p.deg[1] = p.deg[2] = 1;
    for (int v = 0; v < 8; ++v)
        for (int e = 0; e < 8; ++e) {
            // b_v = prod_d (bit ? xi_d : 1 - xi_d): monomial xi^e has coefficient prod_d of
            // (bit, e_d) -> (1,1): 1, (1,0): 0, (0,0): 1, (0,1): -1
            double co = 1.0;
            for (int d = 0; d < 3 && co != 0.0; ++d) {
                const int b = bit(v, d), ed = bit(e, d);
                co *= b ? (ed ? 1.0 : 0.0) : (ed ? -1.0 : 1.0);
            }
            p.c[bit(e, 0)][bit(e, 1)][bit(e, 2)] += co * val[v];
        }
    return p;
}

Poly basis_poly(int v)
{
    double val[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    val[v] = 1.0;
    return trilinear(val);
}

Poly deriv(const Poly &p, int k)
{
    Poly q;
    for (int d = 0; d < 3; ++d) q.deg[d] = p.deg[d];
    q.deg[k] = std::max(0, p.deg[k] - 1);
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c) {
                const int e[3] = {a, b, c};
                if (e[k] == 0) continue;
                int t[3] = {a, b, c};
                t[k] -= 1;
                q.c[t[0]][t[1]][t[2]] += e[k] * p.c[a][b][c];
            }
    return q;
}

Poly mul(const Poly &p, const Poly &q)
{
    Poly r;
    for (int d = 0; d < 3; ++d) r.deg[d] = p.deg[d] + q.deg[d];
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c) {
                const double x = p.c[a][b][c];
                if (x == 0.0) continue;
                for (int u = 0; u <= q.deg[0]; ++u)
                    for (int v = 0; v <= q.deg[1]; ++v)
                        for (int w = 0; w <= q.deg[2]; ++w) r.c[a + u][b + v][c + w] += x * q.c[u][v][w];
            }
    return r;
}

void add_to(Poly &acc, const Poly &p, double s)
{
    for (int d = 0; d < 3; ++d) acc.deg[d] = std::max(acc.deg[d], p.deg[d]);
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c) acc.c[a][b][c] += s * p.c[a][b][c];
}

double eval(const Poly &p, const double xi[3])
{
    double s = 0.0;
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c)
                s += p.c[a][b][c] * std::pow(xi[0], a) * std::pow(xi[1], b) * std::pow(xi[2], c);
    return s;
}

// int_0^1 l_a(xi) xi^m, l_1 = xi, l_0 = 1 - xi
inline double mom1(int a, int m) { return a ? 1.0 / (m + 2) : 1.0 / ((m + 1.0) * (m + 2.0)); }

// int_0^1 l_a(xi) l_b(xi) xi^m
inline double mom2(int a, int b, int m)
{
    if (a && b) return 1.0 / (m + 3);
    if (a || b) return 1.0 / ((m + 2.0) * (m + 3.0));
    return 2.0 / ((m + 1.0) * (m + 2.0) * (m + 3.0));  // int (1-xi)^2 xi^m
}

// int over the cube of b_i p
double int_b(const Poly &p, int i)
{
    double s = 0.0;
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c)
                if (p.c[a][b][c] != 0.0) s += p.c[a][b][c] * mom1(bit(i, 0), a) * mom1(bit(i, 1), b) * mom1(bit(i, 2), c);
    return s;
}

// int over the cube of b_i b_j p
double int_bb(const Poly &p, int i, int j)
{
    double s = 0.0;
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c)
                if (p.c[a][b][c] != 0.0)
                    s += p.c[a][b][c] * mom2(bit(i, 0), bit(j, 0), a) * mom2(bit(i, 1), bit(j, 1), b) *
                         mom2(bit(i, 2), bit(j, 2), c);
    return s;
}

// int over face xi_d = s of b_i b_j p (i, j on the face)
double int_face_bb(const Poly &p, int d, int s, int i, int j)
{
    double tot = 0.0;
    for (int a = 0; a <= p.deg[0]; ++a)
        for (int b = 0; b <= p.deg[1]; ++b)
            for (int c = 0; c <= p.deg[2]; ++c) {
                const int e[3] = {a, b, c};
                if (p.c[a][b][c] == 0.0 || (s == 0 && e[d] > 0)) continue;  // xi_d = 0 kills xi_d^e, e > 0
                double t = p.c[a][b][c];
                for (int ax = 0; ax < 3; ++ax)
                    if (ax != d) t *= mom2(bit(i, ax), bit(j, ax), e[ax]);
                tot += t;
            }
    return tot;
}

Poly cross_comp(const Poly t1[3], const Poly t2[3], int r)
{
    const int u = (r + 1) % 3, v = (r + 2) % 3;
    Poly out = mul(t1[u], t2[v]);
    add_to(out, mul(t1[v], t2[u]), -1.0);
    return out;
}

// Integrals of one cell; false if det J <= 0 at a point of the {0, 1/2, 1}^3 lattice.
bool cell_integrals(const double X[8][3], double &vol, double *Mc, double *Gc, double *Fc)
{
    Poly x[3], t[3][3], cof[3][3];  // t[k][r] = d x_r / d xi_k; cof[k][r] = (t_{k+1} x t_{k+2})_r
    for (int r = 0; r < 3; ++r) {
        double val[8];
        for (int v = 0; v < 8; ++v) val[v] = X[v][r];
        x[r] = trilinear(val);
    }
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) t[k][r] = deriv(x[r], k);
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) cof[k][r] = cross_comp(t[(k + 1) % 3], t[(k + 2) % 3], r);
    Poly det;
    for (int r = 0; r < 3; ++r) add_to(det, mul(t[0][r], cof[0][r]), 1.0);
    for (int p = 0; p < 27; ++p) {
        const double xi[3] = {0.5 * (p % 3), 0.5 * ((p / 3) % 3), 0.5 * (p / 9)};
        if (!(eval(det, xi) > 0.0)) return false;
    }
    vol = 0.0;
    for (int a = 0; a <= det.deg[0]; ++a)
        for (int b = 0; b <= det.deg[1]; ++b)
            for (int c = 0; c <= det.deg[2]; ++c) vol += det.c[a][b][c] / ((a + 1.0) * (b + 1.0) * (c + 1.0));
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) Mc[8 * i + j] = int_bb(det, i, j);
    // (d b_j / d x_d) det J = sum_k cof[k][d] d b_j / d xi_k
    for (int j = 0; j < 8; ++j) {
        const Poly bj = basis_poly(j);
        Poly db[3];
        for (int k = 0; k < 3; ++k) db[k] = deriv(bj, k);
        for (int d = 0; d < 3; ++d) {
            Poly gj;
            for (int k = 0; k < 3; ++k) add_to(gj, mul(cof[k][d], db[k]), 1.0);
            for (int i = 0; i < 8; ++i) Gc[64 * d + 8 * i + j] = int_b(gj, i);
        }
    }
    // outward area-vector density on face xi_d = s: (2s - 1) times cofactor column d
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2, s = f % 2;
        int node[4], n = 0;
        for (int v = 0; v < 8; ++v)
            if (bit(v, d) == s) node[n++] = v;
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 4; ++k)
                for (int l = 0; l < 4; ++l) {
                    const double val = int_face_bb(cof[d][r], d, s, node[k], node[l]);
                    Fc[48 * f + 16 * r + 4 * k + l] = s ? val : -val;
                }
    }
    return true;
}

}  // namespace

int hex_face_node(int f, int k)
{
    const int d = f / 2, s = f % 2;
    int n = 0;
    for (int v = 0; v < 8; ++v)
        if (bit(v, d) == s && n++ == k) return v;
    return -1;
}

tf_status build_hex_mesh(int64_t nv, const double *xyz, int64_t nc, const int32_t *hexes, Mesh &m)
{
    m.nv = nv;
    m.nc = nc;
    m.nf = 6;
    try {
        m.xyz.assign(xyz, xyz + 3 * nv);
        m.hexes.assign(hexes, hexes + 8 * nc);
        m.vol.resize(nc);
        m.hmass.resize(64 * nc);
        m.hgrad.resize(192 * nc);
        m.hface.resize(288 * nc);
        m.normal.resize(18 * nc);
        m.nbr.assign(6 * nc, -1);
        m.nbr_face.assign(6 * nc, -1);
        m.nbr_node.assign(24 * nc, -1);
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "mesh: host allocation failed");
    }
    for (int64_t i = 0; i < 8 * nc; ++i)
        if (hexes[i] < 0 || hexes[i] >= nv)
            return fail(TF_ERR_MESH, "mesh: vertex index out of range in cell " + std::to_string(i / 8));
    // element integrals, cells spread over host threads
    std::atomic<int64_t> bad{-1};
    {
        const unsigned nt = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nc / 256 + 1,
                                                                            std::max(1u, std::thread::hardware_concurrency())));
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                for (int64_t c = t; c < nc; c += nt) {
                    double X[8][3];
                    for (int v = 0; v < 8; ++v)
                        for (int r = 0; r < 3; ++r) X[v][r] = xyz[3 * (int64_t)hexes[8 * c + v] + r];
                    if (!cell_integrals(X, m.vol[c], &m.hmass[64 * c], &m.hgrad[192 * c], &m.hface[288 * c])) {
                        int64_t e = -1;
                        bad.compare_exchange_strong(e, c);
                    }
                }
            });
        for (auto &x : th) x.join();
    }
    if (bad >= 0) return fail(TF_ERR_MESH, "mesh: cell " + std::to_string(bad.load()) + " is inverted or degenerate");
    // integrated face area vectors, canonical: each diagonal runs from its smaller global
    // vertex id to its larger, the diagonal holding the smallest id first; Nbar = 1/2 dA x dB,
    // signed to agree with the cell's own face integral of N
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 6; ++f) {
            int32_t g[4];
            for (int k = 0; k < 4; ++k) g[k] = hexes[8 * c + hex_face_node(f, k)];
            int32_t a0 = std::min(g[0], g[3]), a1 = std::max(g[0], g[3]);
            int32_t b0 = std::min(g[1], g[2]), b1 = std::max(g[1], g[2]);
            if (b0 < a0) {
                std::swap(a0, b0);
                std::swap(a1, b1);
            }
            double dA[3], dB[3];
            for (int r = 0; r < 3; ++r) {
                dA[r] = xyz[3 * (int64_t)a1 + r] - xyz[3 * (int64_t)a0 + r];
                dB[r] = xyz[3 * (int64_t)b1 + r] - xyz[3 * (int64_t)b0 + r];
            }
            const double Nb[3] = {dA[1] * dB[2] - dA[2] * dB[1], dA[2] * dB[0] - dA[0] * dB[2],
                                  dA[0] * dB[1] - dA[1] * dB[0]};
            double own = 0.0;
            for (int r = 0; r < 3; ++r) {
                double sr = 0.0;
                for (int k = 0; k < 16; ++k) sr += m.hface[288 * c + 48 * f + 16 * r + k];
                own += sr * Nb[r];
            }
            const double sg = own < 0.0 ? -0.5 : 0.5;
            for (int r = 0; r < 3; ++r) m.normal[18 * c + 3 * f + r] = sg * Nb[r];
        }
    // face matching on sorted vertex quadruples
    struct Rec {
        int32_t v[4];
        int64_t id;  // 6 * cell + face
    };
    std::vector<Rec> rec;
    try {
        rec.resize(6 * nc);
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "mesh: host allocation failed");
    }
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < 6; ++f) {
            Rec &r = rec[6 * c + f];
            for (int k = 0; k < 4; ++k) r.v[k] = hexes[8 * c + hex_face_node(f, k)];
            std::sort(r.v, r.v + 4);
            r.id = 6 * c + f;
        }
    std::sort(rec.begin(), rec.end(), [](const Rec &a, const Rec &b) {
        for (int k = 0; k < 4; ++k)
            if (a.v[k] != b.v[k]) return a.v[k] < b.v[k];
        return a.id < b.id;
    });
    auto same = [](const Rec &a, const Rec &b) { return std::equal(a.v, a.v + 4, b.v); };
    for (size_t i = 0; i < rec.size();) {
        size_t j = i + 1;
        while (j < rec.size() && same(rec[i], rec[j])) ++j;
        if (j - i > 2) return fail(TF_ERR_MESH, "mesh: a face is shared by more than two cells");
        if (j - i == 2) {
            for (int s = 0; s < 2; ++s) {
                const int64_t id = rec[i + s].id, other = rec[i + 1 - s].id;
                const int64_t c = id / 6, n = other / 6;
                const int f = (int)(id % 6), fn = (int)(other % 6);
                m.nbr[6 * c + f] = (int32_t)n;
                m.nbr_face[6 * c + f] = (int8_t)fn;
                for (int k = 0; k < 4; ++k) {
                    const int32_t gv = hexes[8 * c + hex_face_node(f, k)];
                    for (int v = 0; v < 8; ++v)
                        if (hexes[8 * n + v] == gv) m.nbr_node[24 * c + 4 * f + k] = (int8_t)v;
                }
            }
        }
        i = j;
    }
    return TF_OK;
}

}  // namespace tf
