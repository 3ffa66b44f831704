// Third-order (twenty-node) upwind-DG element on tetrahedra: cell record, device
// element tables and the local solve of one (cell, direction, group) unit.
// Included by sweep_kernel.cuh inside namespace tf, after the PTX helpers.
//
// Nodes: the four vertices, two per edge (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) (first at
// (lambda_a, lambda_b) = (2/3, 1/3)), the four face centres (face f opposite vertex f);
// cubic Lagrange basis on that lattice.  Local system as for the lower orders:
//   [ V sum_k w_k C_k + sigma_t V M + sum_{f inflow} |Omega.N_f| F_f ] psi
//     = V M q + sum_{f inflow} |Omega.N_f| F_f psi_up,       w_k = Omega . grad lambda_k,
// with the exact tables of p3_tables.cpp (M, C_k per unit volume, F per unit area on the
// face's ten nodes).  A 20 x 20 system does not fit a thread's registers: each lane keeps
// its system in shared memory (lane-interleaved, so every access is conflict free) and
// eliminates without pivoting (the symmetric part, (1/2) sum_f |Omega.N_f| F_f + sigma_t V M,
// is positive definite).  One warp per CTA.
#pragma once

template <class T> struct alignas(16) P3Geo {
    int32_t nbr[4];              // neighbour across face f, -1 on the boundary
    T gl[12];                    // grad lambda_k, k = 0..3: (x, y, z)
    T nrm[12];                   // area-weighted outward normal N_f of face f
    T vol;                       // V
    int32_t mat;
    unsigned long long fmap[4];  // face f, face node r (0..9): the neighbour's local node, 5 bits at bit 5 r
};

template <class T> struct P3Dev {
    T M[400];        // int phi_i phi_j / V, row-major
    T C[4][400];     // int phi_i d phi_j / d lambda_k / V
    T F[100];        // int_f phi_r phi_c / A_f on a face's ten nodes (the same for every face)
    int32_t fn[4][10];  // the ten nodes of the face opposite vertex f
};

// shared memory of one lane's system: a(i, j) at [(20 i + j) 32], b_i at [(400 + i) 32]
template <class T> inline size_t p3_warp_bytes() { return (420 * 32 * sizeof(T) + 48 + 127) / 128 * 128; }

template <class T>
__device__ __noinline__ void p3_unit(const SweepArgs<T> &A, const P3Geo<T> *__restrict__ geo,
                                     const P3Dev<T> *__restrict__ tb, T *__restrict__ am, uint32_t e, int g, T ox,
                                     T oy, T oz, size_t psi_dir)
{
    const int G = A.G;
    T *bm = am + 400 * 32;
    const uint32_t c = e >> 4, mask = e & 15u;
    const P3Geo<T> &cg = geo[c];
    T w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = ox * cg.gl[3 * k] + oy * cg.gl[3 * k + 1] + oz * cg.gl[3 * k + 2];
    const T V = cg.vol;
    const T sig = __ldg(A.sigma_t + (size_t)cg.mat * G + g);
    const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 20 * G + g;
    T q[20];
#pragma unroll
    for (int j = 0; j < 20; ++j) q[j] = __ldg(qc + (size_t)j * G);
    for (int i = 0; i < 20; ++i) {
        T bi = T(0);
#pragma unroll
        for (int j = 0; j < 20; ++j) {
            const int ij = 20 * i + j;
            const T m = __ldg(&tb->M[ij]);
            am[ij * 32] = V * (sig * m + w[0] * __ldg(&tb->C[0][ij]) + w[1] * __ldg(&tb->C[1][ij]) +
                               w[2] * __ldg(&tb->C[2][ij]) + w[3] * __ldg(&tb->C[3][ij]));
            bi += m * q[j];
        }
        bm[i * 32] = V * bi;
    }
    T *psi = reinterpret_cast<T *>(A.psi);
    for (int f = 0; f < 4; ++f) {
        if (!((mask >> f) & 1u)) continue;
        const T s = fabs(ox * cg.nrm[3 * f] + oy * cg.nrm[3 * f + 1] + oz * cg.nrm[3 * f + 2]);
        int fn[10];
#pragma unroll
        for (int r = 0; r < 10; ++r) fn[r] = __ldg(&tb->fn[f][r]);
#pragma unroll
        for (int r = 0; r < 10; ++r)
#pragma unroll
            for (int k = 0; k < 10; ++k) am[(20 * fn[r] + fn[k]) * 32] += s * __ldg(&tb->F[10 * r + k]);
        const int n = cg.nbr[f];
        if (n < 0) continue;  // vacuum boundary: no inflow
        const unsigned long long fm = cg.fmap[f];
        T up[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            const uint32_t node = (uint32_t)(fm >> (5 * k)) & 31u;
            up[k] = __ldcg(psi + ((psi_dir + (size_t)n) * 20 + node) * G + g);
        }
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            T t = T(0);
#pragma unroll
            for (int k = 0; k < 10; ++k) t += __ldg(&tb->F[10 * r + k]) * up[k];
            bm[fn[r] * 32] += s * t;
        }
    }
    // Gaussian elimination without pivoting; the diagonal keeps the pivots' reciprocals
    for (int k = 0; k < 20; ++k) {
        const T r = rcp(am[21 * k * 32]);
        const T bk = bm[k * 32];
        for (int i = k + 1; i < 20; ++i) {
            const T l = am[(20 * i + k) * 32] * r;
            for (int j = k + 1; j < 20; ++j) am[(20 * i + j) * 32] -= l * am[(20 * k + j) * 32];
            bm[i * 32] -= l * bk;
        }
        am[21 * k * 32] = r;
    }
    T *out = psi + (psi_dir + c) * 20 * (size_t)G + g;
    for (int i = 19; i >= 0; --i) {
        T s = bm[i * 32];
        for (int j = i + 1; j < 20; ++j) s -= am[(20 * i + j) * 32] * bm[j * 32];
        s *= am[21 * i * 32];
        bm[i * 32] = s;
        out[(size_t)i * G] = s;
    }
}

// A task: lanes over the (cell, group) units of its cells (one t-level, independent).
template <class T>
__device__ __forceinline__ void run_task_p3(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz, size_t psi_dir,
                                            unsigned char *wsm)
{
    const P3Geo<T> *geo = reinterpret_cast<const P3Geo<T> *>(A.geo2);
    const P3Dev<T> *tb = reinterpret_cast<const P3Dev<T> *>(A.p3tab);
    T *am = reinterpret_cast<T *>(wsm) + lane;
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t nu = ncell * (uint32_t)A.G;
    for (uint32_t u = lane; u < nu; u += 32) {
        const uint32_t k = u / (uint32_t)A.G;
        const int g = (int)(u - k * (uint32_t)A.G);
        p3_unit(A, geo, tb, am, __ldg(A.cells + ti.x + k), g, ox, oy, oz, psi_dir);
    }
}
