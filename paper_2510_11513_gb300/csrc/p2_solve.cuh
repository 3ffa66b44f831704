// Second-order (ten-node) upwind-DG element on tetrahedra: cell record, exact
// element tables and the local solve of one (cell, direction, group) unit.
// Included by sweep_kernel.cuh inside namespace tf.
//
// Nodes of a cell: its four vertices (caller's local order), then the midpoints
// of the local edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).  Basis (barycentric
// lambda): vertex v: lambda_v (2 lambda_v - 1); edge (a,b): 4 lambda_a lambda_b.
// Local system (weak form of Eq. (1) integrated back by parts, upwind trace on
// inflow faces, as for the linear element):
//   [ K(Omega) + sigma_t V Mh + sum_{f inflow} |Omega.N_f| Fh_f ] psi
//     = V Mh q + sum_{f inflow} |Omega.N_f| Fh_f psi_up
// with Mh = int phi_i phi_j / V, Fh_f = int_f phi_i phi_j / A_f and
// K_ij = int phi_i Omega.grad phi_j; writing w_k = Omega.grad lambda_k,
// P_im = int phi_i lambda_m / V and p_i = int phi_i / V:
//   vertex j = v:      K_iv = V w_v (4 P_iv - p_i)
//   edge j = (a,b):    K_ie = 4 V (w_a P_ib + w_b P_ia).
// The tables are exact rationals from int lambda^a = 6 V a! / (|a| + 3)! on the
// cell and 2 A a! / (|a| + 2)! on a face.  The symmetric part of the matrix is
// (1/2) sum_f |Omega.N_f| Fh_f + sigma_t V Mh, positive definite, so Gaussian
// elimination needs no pivoting.
#pragma once

#include "p2_tables.h"

template <class T> struct alignas(16) P2Geo {
    T gl[12];          // grad lambda_k, k = 0..3: (x, y, z)
    T nrm[12];         // area-weighted outward normal N_f of face f (opposite vertex f)
    T vol;             // V
    int32_t mat;
    int32_t nbr[4];    // neighbour across face f, -1 on the boundary
    uint32_t fmap[3];  // face f, face node b: the neighbour's local node, 4 bits at bit 24 f + 4 b
};

// 10 x 10 Gaussian elimination without pivoting (positive definite symmetric part).
template <class T> __device__ __forceinline__ void p2_solve10(T a[10][10], T b[10], T x[10])
{
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const T r = rcp(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < 10; ++i) {
            const T l = a[i][k] * r;
#pragma unroll
            for (int j = k + 1; j < 10; ++j) a[i][j] -= l * a[k][j];
            b[i] -= l * b[k];
        }
        a[k][k] = r;
    }
#pragma unroll
    for (int i = 9; i >= 0; --i) {
        T s = b[i];
#pragma unroll
        for (int j = i + 1; j < 10; ++j) s -= a[i][j] * x[j];
        x[i] = s * a[i][i];
    }
}

// One unit: cell entry e = (cell << 4) | inflow mask (caller's face order), group g.
// q and psi are node-major per cell: [cell][node][G].  Upwind rows were written by
// other warps in this launch and are read through L2.
template <class T>
__device__ __forceinline__ void p2_unit(const SweepArgs<T> &A, const P2Geo<T> *__restrict__ geo, uint32_t e, int g,
                                        T ox, T oy, T oz, size_t psi_dir)
{
    const int G = A.G;
    const uint32_t c = e >> 4, mask = e & 15u;
    const P2Geo<T> &cg = geo[c];
    T w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = ox * __ldg(&cg.gl[3 * k]) + oy * __ldg(&cg.gl[3 * k + 1]) + oz * __ldg(&cg.gl[3 * k + 2]);
    const T V = __ldg(&cg.vol);
    const T sig = __ldg(A.sigma_t + (size_t)__ldg(&cg.mat) * G + g);
    const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 10 * G + g;
    T q[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) q[j] = __ldg(qc + (size_t)j * G);
    T a[10][10], b[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        T bi = T(0);
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            T kij;
            if (j < 4) {
                kij = w[j] * T(4.0 * p2_P(i, j) - p2_p(i));
            } else {
                const int ea = p2_edge_end(j - 4, 0), eb = p2_edge_end(j - 4, 1);
                kij = T(4.0 * p2_P(i, eb)) * w[ea] + T(4.0 * p2_P(i, ea)) * w[eb];
            }
            a[i][j] = V * (sig * T(p2_M(i, j)) + kij);
            bi += T(p2_M(i, j)) * q[j];
        }
        b[i] = V * bi;
    }
    T *psi = reinterpret_cast<T *>(A.psi);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!((mask >> f) & 1u)) continue;
        const T s = fabs(ox * __ldg(&cg.nrm[3 * f]) + oy * __ldg(&cg.nrm[3 * f + 1]) + oz * __ldg(&cg.nrm[3 * f + 2]));
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int k = 0; k < 6; ++k) a[p2_face_node(f, r)][p2_face_node(f, k)] += s * T(p2_F(r, k));
        const int n = __ldg(&cg.nbr[f]);
        if (n < 0) continue;  // vacuum boundary: no inflow
        T up[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int bit = 24 * f + 4 * k;
            const uint32_t m = (__ldg(&cg.fmap[bit >> 5]) >> (bit & 31)) & 15u;
            up[k] = __ldcg(psi + ((psi_dir + (size_t)n) * 10 + m) * G + g);
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            T t = T(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) t += T(p2_F(r, k)) * up[k];
            b[p2_face_node(f, r)] += s * t;
        }
    }
    T x[10];
    p2_solve10(a, b, x);
    T *out = psi + (psi_dir + c) * 10 * (size_t)G + g;
#pragma unroll
    for (int i = 0; i < 10; ++i) out[(size_t)i * G] = x[i];
}

// A task: lanes over the (cell, group) units of its cells (one t-level, independent).
template <class T>
__device__ __forceinline__ void run_task_p2(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz, size_t psi_dir)
{
    const P2Geo<T> *geo = reinterpret_cast<const P2Geo<T> *>(A.geo2);
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t nu = ncell * (uint32_t)A.G;
    for (uint32_t u = lane; u < nu; u += 32) {
        const uint32_t k = u / (uint32_t)A.G;
        const int g = (int)(u - k * (uint32_t)A.G);
        p2_unit(A, geo, __ldg(A.cells + ti.x + k), g, ox, oy, oz, psi_dir);
    }
}
