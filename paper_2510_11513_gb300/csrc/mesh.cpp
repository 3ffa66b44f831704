// Host geometry of the tetrahedral mesh and the angular quadrature.
//
// Geometry is FP64 and compiled without floating-point contraction, so the
// face normals and hence the face classification (and the sweep graph built
// from it) are reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "tf_internal.h"

namespace tf {

namespace {

inline void sorted3(int32_t a, int32_t b, int32_t c, int32_t out[3])
{
    if (a > b) std::swap(a, b);
    if (b > c) std::swap(b, c);
    if (a > b) std::swap(a, b);
    out[0] = a;
    out[1] = b;
    out[2] = c;
}

}  // namespace

// Volumes, basis gradients, area-weighted outward normals and face neighbours.
// Basis function b_j of a linear tetrahedron has a constant gradient: rows of
// the inverse of J = [x1-x0, x2-x0, x3-x0] for j = 1..3 and minus their sum
// for j = 0 (these give the f_i df_j/dx det J element integrals of Table
// Table 1 as (V/4) d b_j / dx).  Face f is opposite local vertex f; its
// normal is (1/2)(xb - xa) x (xc - xa) over the face's global vertices in
// increasing index order, flipped to point away from vertex f, so the two
// cells sharing a face hold exactly opposite normals.
tf_status build_mesh(int64_t nv, const double *xyz, int64_t nc, const int32_t *tets, Mesh &m)
{
    m.nv = nv;
    m.nc = nc;
    try {
        m.xyz.assign(xyz, xyz + 3 * nv);
        m.tets.assign(tets, tets + 4 * nc);
        m.vol.resize(nc);
        m.grad.resize(12 * nc);
        m.normal.resize(12 * nc);
        m.nbr.assign(4 * nc, -1);
        m.nbr_face.assign(4 * nc, -1);
        m.nbr_node.assign(16 * nc, -1);
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "mesh: host allocation failed");
    }
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t *t = tets + 4 * c;
        for (int i = 0; i < 4; ++i)
            if (t[i] < 0 || t[i] >= nv) return fail(TF_ERR_MESH, "mesh: vertex index out of range in cell " + std::to_string(c));
        const double *x0 = xyz + 3 * (int64_t)t[0];
        double J[3][3];
        for (int k = 0; k < 3; ++k)
            for (int r = 0; r < 3; ++r) J[r][k] = xyz[3 * (int64_t)t[k + 1] + r] - x0[r];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0)) return fail(TF_ERR_MESH, "mesh: cell " + std::to_string(c) + " is inverted or degenerate");
        m.vol[c] = det / 6.0;
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
        double *g = &m.grad[12 * c];
        for (int d = 0; d < 3; ++d) {
            g[3 + d] = inv[0][d];
            g[6 + d] = inv[1][d];
            g[9 + d] = inv[2][d];
            g[d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
        }
        for (int f = 0; f < 4; ++f) {
            int32_t s[3];
            sorted3(t[(f + 1) & 3], t[(f + 2) & 3], t[(f + 3) & 3], s);
            const double *xa = xyz + 3 * (int64_t)s[0], *xb = xyz + 3 * (int64_t)s[1], *xc = xyz + 3 * (int64_t)s[2];
            const double e1[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
            const double e2[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
            double N[3] = {0.5 * (e1[1] * e2[2] - e1[2] * e2[1]), 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]),
                           0.5 * (e1[0] * e2[1] - e1[1] * e2[0])};
            const double *xo = xyz + 3 * (int64_t)t[f];
            const double side = (N[0] * (xo[0] - xa[0]) + N[1] * (xo[1] - xa[1])) + N[2] * (xo[2] - xa[2]);
            if (side > 0.0) {
                N[0] = -N[0];
                N[1] = -N[1];
                N[2] = -N[2];
            }
            double *out = &m.normal[12 * c + 3 * f];
            out[0] = N[0];
            out[1] = N[1];
            out[2] = N[2];
        }
    }
    // Face matching: order face records by their sorted vertex triple.
    struct Rec {
        int32_t v[3];
        int64_t id;  // 4 * cell + face
    };
    std::vector<Rec> rec;
    try {
        rec.resize(4 * nc);
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "mesh: host allocation failed");
    }
    for (int64_t c = 0; c < nc; ++c) {
        const int32_t *t = tets + 4 * c;
        for (int f = 0; f < 4; ++f) {
            Rec &r = rec[4 * c + f];
            sorted3(t[(f + 1) & 3], t[(f + 2) & 3], t[(f + 3) & 3], r.v);
            r.id = 4 * c + f;
        }
    }
    std::sort(rec.begin(), rec.end(), [](const Rec &a, const Rec &b) {
        if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
        if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
        if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
        return a.id < b.id;
    });
    auto same = [](const Rec &a, const Rec &b) { return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2]; };
    for (size_t i = 0; i < rec.size();) {
        size_t j = i + 1;
        while (j < rec.size() && same(rec[i], rec[j])) ++j;
        if (j - i > 2) return fail(TF_ERR_MESH, "mesh: a face is shared by more than two cells");
        if (j - i == 2) {
            for (int s = 0; s < 2; ++s) {
                const int64_t id = rec[i + s].id, other = rec[i + 1 - s].id;
                const int64_t c = id >> 2, n = other >> 2;
                const int f = (int)(id & 3), fn = (int)(other & 3);
                m.nbr[4 * c + f] = (int32_t)n;
                m.nbr_face[4 * c + f] = (int8_t)fn;
                for (int a = 0; a < 4; ++a) {
                    if (a == f) continue;
                    for (int b = 0; b < 4; ++b)
                        if (tets[4 * n + b] == tets[4 * c + a]) m.nbr_node[16 * c + 4 * f + a] = (int8_t)b;
                }
            }
        }
        i = j;
    }
    return TF_OK;
}

// Gauss-Legendre cosines by Newton's method on P_n (three-term recurrence),
// times equispaced half-offset azimuths: the product S_N set whose weights
// sum to 4 pi (Eq. (2) discretised).
tf_status build_quadrature(int32_t n_polar, int32_t n_az, Quad &q)
{
    if (n_polar < 1 || n_az < 1 || (int64_t)n_polar * n_az > 65535)
        return fail(TF_ERR_ARG, "quadrature: need n_polar, n_azimuthal >= 1 and at most 65535 directions");
    const int n = n_polar;
    std::vector<double> mu(n), wm(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z = z - dz;
            if (std::fabs(dz) <= 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 1; k < n; ++k) {
            const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        mu[n - 1 - i] = z;
        wm[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    q.D = n_polar * n_az;
    q.omega.resize(3 * (size_t)q.D);
    q.w.resize(q.D);
    for (int i = 0; i < n_polar; ++i) {
        const double s = std::sqrt(1.0 - mu[i] * mu[i]);
        for (int k = 0; k < n_az; ++k) {
            const double ph = (k + 0.5) * (2.0 * M_PI / n_az);
            const int a = i * n_az + k;
            q.omega[3 * a + 0] = s * std::cos(ph);
            q.omega[3 * a + 1] = s * std::sin(ph);
            q.omega[3 * a + 2] = mu[i];
            q.w[a] = wm[i] * (2.0 * M_PI / n_az);
        }
    }
    return TF_OK;
}

}  // namespace tf
