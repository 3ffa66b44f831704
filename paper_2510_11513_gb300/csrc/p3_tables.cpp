// Exact element tables of the third-order (twenty-node) tetrahedron, computed on
// the host once: the cubic Lagrange basis on the equispaced lattice lambda = alpha/3,
// phi_alpha = prod_k prod_{m < alpha_k} (3 lambda_k - m) / (m + 1), expanded into
// monomials in the barycentric coordinates and integrated exactly with
//   int_K lambda^a dV / V = 6 a! / (|a| + 3)!,   int_F lambda^a dA / A = 2 a! / (|a| + 2)!
// (a! = product of the exponents' factorials; on the face opposite vertex f, a_f = 0).
// Node order: vertices 0..3; two nodes per edge (0,1) (0,2) (0,3) (1,2) (1,3) (2,3),
// first at (lambda_a, lambda_b) = (2/3, 1/3), then (1/3, 2/3); face centres 16 + f.
#include <array>
#include <map>
#include <vector>

#include "tf_internal.h"

namespace tf {

namespace {

using Exps = std::array<int, 4>;
using Poly = std::map<Exps, double>;

Poly mul(const Poly &a, const Poly &b)
{
    Poly out;
    for (const auto &x : a)
        for (const auto &y : b) {
            Exps e;
            for (int k = 0; k < 4; ++k) e[k] = x.first[k] + y.first[k];
            out[e] += x.second * y.second;
        }
    return out;
}

Poly dpoly(const Poly &p, int k)
{
    Poly out;
    for (const auto &x : p) {
        if (x.first[k] == 0) continue;
        Exps e = x.first;
        e[k] -= 1;
        out[e] += x.second * x.first[k];
    }
    return out;
}

double fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

double integrate_cell(const Poly &p)
{
    double s = 0.0;
    for (const auto &x : p) {
        const Exps &e = x.first;
        s += x.second * 6.0 * fact(e[0]) * fact(e[1]) * fact(e[2]) * fact(e[3]) / fact(e[0] + e[1] + e[2] + e[3] + 3);
    }
    return s;
}

double integrate_face(const Poly &p, int f)
{
    double s = 0.0;
    for (const auto &x : p) {
        const Exps &e = x.first;
        if (e[f] != 0) continue;
        s += x.second * 2.0 * fact(e[0]) * fact(e[1]) * fact(e[2]) * fact(e[3]) / fact(e[0] + e[1] + e[2] + e[3] + 2);
    }
    return s;
}

}  // namespace

void p3_node_alpha(int i, int al[4])
{
    static const int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    al[0] = al[1] = al[2] = al[3] = 0;
    if (i < 4) {
        al[i] = 3;
    } else if (i < 16) {
        const int e = (i - 4) / 2, second = (i - 4) % 2;
        al[E[e][0]] = second ? 1 : 2;
        al[E[e][1]] = second ? 2 : 1;
    } else {
        for (int k = 0; k < 4; ++k) al[k] = k == i - 16 ? 0 : 1;
    }
}

void p3_element_tables(P3Tables &t)
{
    std::vector<Poly> B(20);
    for (int i = 0; i < 20; ++i) {
        int al[4];
        p3_node_alpha(i, al);
        Poly p;
        p[Exps{0, 0, 0, 0}] = 1.0;
        for (int k = 0; k < 4; ++k)
            for (int m = 0; m < al[k]; ++m) {
                Poly fac;
                Exps e{0, 0, 0, 0};
                e[k] = 1;
                fac[e] = 3.0 / (m + 1);
                if (m > 0) fac[Exps{0, 0, 0, 0}] = -double(m) / (m + 1);
                p = mul(p, fac);
            }
        B[i] = p;
    }
    for (int i = 0; i < 20; ++i) {
        t.p[i] = integrate_cell(B[i]);
        for (int j = 0; j < 20; ++j) {
            t.M[i * 20 + j] = integrate_cell(mul(B[i], B[j]));
            for (int k = 0; k < 4; ++k) t.C[k][i * 20 + j] = integrate_cell(mul(B[i], dpoly(B[j], k)));
        }
    }
    for (int f = 0; f < 4; ++f) {
        int n = 0;
        for (int i = 0; i < 20; ++i) {
            int al[4];
            p3_node_alpha(i, al);
            if (al[f] == 0) t.fn[f][n++] = i;  // the face's nodes, in node order
        }
        for (int r = 0; r < 10; ++r) {
            Poly one;
            one[Exps{0, 0, 0, 0}] = 1.0;
            t.fav[f][r] = integrate_face(mul(B[t.fn[f][r]], one), f);
            for (int c = 0; c < 10; ++c) t.F[f][r * 10 + c] = integrate_face(mul(B[t.fn[f][r]], B[t.fn[f][c]]), f);
        }
    }
}

}  // namespace tf
