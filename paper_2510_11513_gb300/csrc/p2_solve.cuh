// Second-order (ten-node) upwind-DG element on tetrahedra: cell record, exact
// element tables and the local solve of one (cell, direction, group) unit.
// Included by sweep_kernel.cuh inside namespace tf, after the PTX helpers.
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
    int32_t nbr[4];    // neighbour across face f, -1 on the boundary (16-byte aligned: read as one int4)
    T gl[12];          // grad lambda_k, k = 0..3: (x, y, z)
    T nrm[12];         // area-weighted outward normal N_f of face f (opposite vertex f)
    T vol;             // V
    int32_t mat;
    uint32_t fmap[3];  // face f, face node b: the neighbour's local node, 4 bits at bit 24 f + 4 b
};
static_assert(offsetof(P2Geo<float>, nbr) % 16 == 0 && offsetof(P2Geo<double>, nbr) % 16 == 0,
              "second-order neighbour list must be 16-byte aligned");
static_assert(sizeof(P2Geo<float>) % 16 == 0 && sizeof(P2Geo<double>) % 16 == 0,
              "second-order records must be whole 16-byte units (bulk copies)");

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

// The local system of one unit from its inputs and its solution x: cg the cell
// record, mask its inflow faces (caller's order), q(j) the source at node j,
// up(f, k) the upwind value at face node k of interior inflow face f.
template <class T, class Q, class Up>
__device__ __forceinline__ void p2_local_solve(const P2Geo<T> &cg, uint32_t mask, T sig, T ox, T oy, T oz, Q q, Up up,
                                               T x[10])
{
    T w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = ox * cg.gl[3 * k] + oy * cg.gl[3 * k + 1] + oz * cg.gl[3 * k + 2];
    const T V = cg.vol;
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
            bi += T(p2_M(i, j)) * q(j);
        }
        b[i] = V * bi;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!((mask >> f) & 1u)) continue;
        const T s = fabs(ox * cg.nrm[3 * f] + oy * cg.nrm[3 * f + 1] + oz * cg.nrm[3 * f + 2]);
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int k = 0; k < 6; ++k) a[p2_face_node(f, r)][p2_face_node(f, k)] += s * T(p2_F(r, k));
        if (cg.nbr[f] < 0) continue;  // vacuum boundary: no inflow
        T u[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) u[k] = up(f, k);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            T t = T(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) t += T(p2_F(r, k)) * u[k];
            b[p2_face_node(f, r)] += s * t;
        }
    }
    p2_solve10(a, b, x);
}

// Neighbour's local node of face node k of face f.
template <class T> __device__ __forceinline__ uint32_t p2_fmap(const P2Geo<T> &cg, int f, int k)
{
    const int bit = 24 * f + 4 * k;
    return (cg.fmap[bit >> 5] >> (bit & 31)) & 15u;
}

// One unit read straight from global memory: cell entry e = (cell << 4) | inflow
// mask (caller's face order), group g.  q and psi are node-major per cell,
// [cell][node][G]; upwind rows were written by other warps in this launch and are
// read through L2.
template <class T>
__device__ __forceinline__ void p2_unit(const SweepArgs<T> &A, const P2Geo<T> *__restrict__ geo, uint32_t e, int g,
                                        T ox, T oy, T oz, size_t psi_dir)
{
    const int G = A.G;
    const uint32_t c = e >> 4;
    const P2Geo<T> &cg = geo[c];
    const T sig = __ldg(A.sigma_t + (size_t)cg.mat * G + g);
    const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 10 * G + g;
    T *psi = reinterpret_cast<T *>(A.psi);
    T x[10];
    p2_local_solve(
        cg, e & 15u, sig, ox, oy, oz, [&](int j) { return __ldg(qc + (size_t)j * G); },
        [&](int f, int k) {
            return __ldcg(psi + ((psi_dir + (size_t)cg.nbr[f]) * 10 + p2_fmap(cg, f, k)) * G + g);
        },
        x);
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

// Staged variant (FP32, G a multiple of 32, at most 32 cells per task): lanes over
// groups, one cell at a time; the cell record, its source row [10][G] and the six
// face-node rows [G] of each interior inflow neighbour are copied into shared
// memory by bulk asynchronous copies one cell ahead (two stages per warp), so the
// solve of one cell overlaps the loads of the next.  Stage layout: record, q row,
// up to 18 upwind node rows (inflow faces in face order, face nodes in face order).
__host__ __device__ constexpr uint32_t p2_stage_bytes(int G) { return 144u + 112u * (uint32_t)G; }

__device__ __forceinline__ bool run_task_p2_staged(const SweepArgs<float> &A, uint4 ti, int lane, float ox, float oy,
                                                   float oz, size_t psi_dir, unsigned char *wsm, uint64_t *bars,
                                                   uint32_t &ph, unsigned long long *wacc)
{
    static_assert(sizeof(P2Geo<float>) == 144, "second-order float record is 144 bytes");
    const unsigned FULL = 0xffffffffu;
    const int G = A.G;
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t row = (uint32_t)G * 4u, stage = p2_stage_bytes(G);
    const P2Geo<float> *geo = reinterpret_cast<const P2Geo<float> *>(A.geo2);
    // each lane reads the neighbours and face-node maps of "its" cell of the task
    const uint32_t e_l = lane < (int)ncell ? __ldg(A.cells + ti.x + lane) : 0u;
    int4 n_l = make_int4(-1, -1, -1, -1);
    uint32_t f0 = 0, f1 = 0, f2 = 0;
    if (lane < (int)ncell) {
        const P2Geo<float> &cg = geo[e_l >> 4];
        n_l = __ldg(reinterpret_cast<const int4 *>(cg.nbr));
        f0 = __ldg(&cg.fmap[0]);
        f1 = __ldg(&cg.fmap[1]);
        f2 = __ldg(&cg.fmap[2]);
    }
    if (lane == 0) fence_proxy_async_global();  // psi rows of other warps, acquired through the queue
    const float *psi_g = reinterpret_cast<const float *>(A.psi);
    auto issue = [&](uint32_t k) {
        const int src = (int)k;
        const uint32_t ek = __shfl_sync(FULL, e_l, src);
        int4 nb;
        nb.x = __shfl_sync(FULL, n_l.x, src);
        nb.y = __shfl_sync(FULL, n_l.y, src);
        nb.z = __shfl_sync(FULL, n_l.z, src);
        nb.w = __shfl_sync(FULL, n_l.w, src);
        const uint32_t fm0 = __shfl_sync(FULL, f0, src), fm1 = __shfl_sync(FULL, f1, src),
                       fm2 = __shfl_sync(FULL, f2, src);
        const uint32_t s = k & 1u, mask = ek & 15u, c = ek >> 4;
        const uint32_t upm = (((mask & 1u) && nb.x >= 0) ? 1u : 0u) | (((mask & 2u) && nb.y >= 0) ? 2u : 0u) |
                             (((mask & 4u) && nb.z >= 0) ? 4u : 0u) | (((mask & 8u) && nb.w >= 0) ? 8u : 0u);
        const uint32_t n_rows = 6u * (uint32_t)__popc(upm);
        unsigned char *st = wsm + s * stage;
        fence_proxy_async_shared();  // this lane's generic reads of the stage (cell k - 2) before async writes
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[s], 144u + 10u * row);
            mbar_arrive_expect_tx(&bars[3 + s], n_rows * row);
        }
        __syncwarp();
        if (lane == 0) {
            bulk_g2s(st, geo + c, 144u, &bars[s]);
        } else if (lane == 1) {
            bulk_g2s(st + 144, reinterpret_cast<const float *>(A.q) + (size_t)c * 10 * G, 10u * row, &bars[s]);
        } else if (lane < 2 + (int)n_rows) {
            const int t = lane - 2, slot = t / 6, kk = t - 6 * slot;
            uint32_t m = upm;
            for (int r = 0; r < slot; ++r) m &= m - 1u;  // the slot-th interior inflow face
            const int f = __ffs(m) - 1;
            const int nbf = f == 0 ? nb.x : (f == 1 ? nb.y : (f == 2 ? nb.z : nb.w));
            const int bit = 24 * f + 4 * kk;
            const uint32_t word = (bit >> 5) == 0 ? fm0 : ((bit >> 5) == 1 ? fm1 : fm2);
            const uint32_t node = (word >> (bit & 31)) & 15u;
            bulk_g2s(st + 144 + 10 * row + (uint32_t)t * row, psi_g + ((psi_dir + (size_t)nbf) * 10 + node) * G, row,
                     &bars[3 + s]);
        }
    };
    issue(0);
    float *psi = reinterpret_cast<float *>(A.psi);
    for (uint32_t k = 0; k < ncell; ++k) {
        const uint32_t s = k & 1u;
        if (k + 1 < ncell) issue(k + 1);
        if (!mbar_wait(&bars[s], (ph >> s) & 1u, A.wait_limit_ns, &A.ctrl->error, wacc)) return false;
        ph ^= 1u << s;
        if (!mbar_wait(&bars[3 + s], (ph >> (3 + s)) & 1u, A.wait_limit_ns, &A.ctrl->error, wacc)) return false;
        ph ^= 1u << (3 + s);
        const unsigned char *st = wsm + s * stage;
        const P2Geo<float> &cg = *reinterpret_cast<const P2Geo<float> *>(st);
        const float *qs = reinterpret_cast<const float *>(st + 144);
        const float *us = reinterpret_cast<const float *>(st + 144 + 10 * row);
        const uint32_t ek = __shfl_sync(FULL, e_l, (int)k);
        const uint32_t mask = ek & 15u, c = ek >> 4;
        // slot of each interior inflow face among the staged upwind rows
        uint32_t upm = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) upm |= (((mask >> f) & 1u) && cg.nbr[f] >= 0 ? 1u : 0u) << f;
        for (int g = lane; g < G; g += 32) {
            const float sig = __ldg(A.sigma_t + (size_t)cg.mat * G + g);
            float x[10];
            p2_local_solve(
                cg, mask, sig, ox, oy, oz, [&](int j) { return qs[j * G + g]; },
                [&](int f, int kk) { return us[(6 * __popc(upm & ((1u << f) - 1u)) + kk) * G + g]; }, x);
            float *out = psi + (psi_dir + c) * 10 * (size_t)G + g;
#pragma unroll
            for (int i = 0; i < 10; ++i) out[(size_t)i * G] = x[i];
        }
        __syncwarp();
    }
    return true;
}
