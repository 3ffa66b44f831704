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
// face's ten nodes).  A 20 x 20 system does not fit one thread's registers, so four
// lanes share a unit: lane s of the four holds rows 4 r + s (r = 0..4) of the matrix and
// right-hand side in registers, the pivot row is broadcast inside the four with shuffles,
// and every lane updates its own rows (Gaussian elimination without pivoting: the
// symmetric part, (1/2) sum_f |Omega.N_f| F_f + sigma_t V M, is positive definite).
// A warp solves eight units at a time.
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
    T M[400];           // int phi_i phi_j / V, row-major
    T C[4][400];        // int phi_i d phi_j / d lambda_k / V
    T F[100];           // int_f phi_r phi_c / A_f on a face's ten nodes (the same for every face)
    int32_t fn[4][10];  // the ten nodes of the face opposite vertex f
    T FA[4][400];       // F of face f placed in the 20 x 20 matrix (zero off the face's nodes)
    T FU[4][200];       // [f][i][c]: F(r, c) for the row i = fn[f][r] of the face, zero elsewhere
};

// lattice index of node i in coordinate k (compile-time structure of the element)
__host__ __device__ constexpr int p3_alpha(int i, int k)
{
    constexpr int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    if (i < 4) return i == k ? 3 : 0;
    if (i < 16) {
        const int e = (i - 4) / 2, second = (i - 4) % 2;
        return E[e][0] == k ? (second ? 1 : 2) : (E[e][1] == k ? (second ? 2 : 1) : 0);
    }
    return k == i - 16 ? 0 : 1;
}

// the r-th node (node order) of the face opposite vertex f
__host__ __device__ constexpr int p3_face_node(int f, int r)
{
    int n = 0;
    for (int i = 0; i < 20; ++i)
        if (p3_alpha(i, f) == 0) {
            if (n == r) return i;
            ++n;
        }
    return -1;
}


// One unit on four lanes: sub = lane & 3 (rows 4 r + sub), the unit's cell entry e and group g.
template <class T>
__device__ __forceinline__ void p3_unit4(const SweepArgs<T> &A, const P3Geo<T> *__restrict__ geo,
                                         const P3Dev<T> *__restrict__ tb, int sub, bool live, uint32_t e, int g,
                                         T ox, T oy, T oz, size_t psi_dir)
{
    const unsigned FULL = 0xffffffffu;
    const int G = A.G;
    const uint32_t c = e >> 4, mask = e & 15u;
    const P3Geo<T> &cg = geo[c];
    T w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = ox * cg.gl[3 * k] + oy * cg.gl[3 * k + 1] + oz * cg.gl[3 * k + 2];
    const T V = cg.vol;
    const T sig = live ? __ldg(A.sigma_t + (size_t)cg.mat * G + g) : T(1);
    const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 20 * G + g;
    T q[20];
#pragma unroll
    for (int j = 0; j < 20; ++j) q[j] = live ? __ldg(qc + (size_t)j * G) : T(0);
    // rows 4 r + sub: A = V (sigma_t M + sum_k w_k C_k); C_k(i, j) vanishes unless node j's
    // lattice index has k, so each entry takes one to three streaming terms
    T a[5][20], b[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int i = 4 * r + sub;
        T bi = T(0);
#pragma unroll
        for (int j = 0; j < 20; ++j) {
            const T m = __ldg(&tb->M[20 * i + j]);
            T kij = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (p3_alpha(j, k) > 0) kij += w[k] * __ldg(&tb->C[k][20 * i + j]);
            a[r][j] = V * (sig * m + kij);
            bi += m * q[j];
        }
        b[r] = V * bi;
    }
    T *psi = reinterpret_cast<T *>(A.psi);
    // inflow faces (one loop body for all four, to keep the kernel's code small): the face
    // matrices come expanded to the lane's rows from the tables
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        if (!((mask >> f) & 1u)) continue;
        const T s = fabs(ox * cg.nrm[3 * f] + oy * cg.nrm[3 * f + 1] + oz * cg.nrm[3 * f + 2]);
        const int n = cg.nbr[f];
        T up[10];
        if (n >= 0 && live) {
            const unsigned long long fm = cg.fmap[f];
#pragma unroll
            for (int k = 0; k < 10; ++k)
                up[k] = __ldcg(psi + ((psi_dir + (size_t)n) * 20 + ((uint32_t)(fm >> (5 * k)) & 31u)) * G + g);
        } else {
#pragma unroll
            for (int k = 0; k < 10; ++k) up[k] = T(0);  // vacuum boundary: no inflow
        }
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const int i = 4 * r + sub;
            const T *fa = &tb->FA[f][20 * i];
            const T *fu = &tb->FU[f][10 * i];
#pragma unroll
            for (int j = 0; j < 20; ++j) a[r][j] += s * __ldg(fa + j);
            T t = T(0);
#pragma unroll
            for (int cc = 0; cc < 10; ++cc) t += __ldg(fu + cc) * up[cc];
            b[r] += s * t;
        }
    }
    // elimination: the pivot row k lives in lane (k & 3) of the four, local row k >> 2
    T x[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) {
        const int owner = k & 3, rk = k >> 2;
        T pv[20];
#pragma unroll
        for (int j = k; j < 20; ++j) pv[j] = __shfl_sync(FULL, a[rk][j], owner, 4);
        const T pb = __shfl_sync(FULL, b[rk], owner, 4);
        const T rp = rcp(pv[k]);
        if (sub == owner) a[rk][k] = rp;  // the owner keeps the reciprocal for the back substitution
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            if (4 * r + sub <= k) continue;  // rows at or above the pivot are finished
            const T l = a[r][k] * rp;
#pragma unroll
            for (int j = k + 1; j < 20; ++j) a[r][j] -= l * pv[j];
            b[r] -= l * pb;
        }
    }
#pragma unroll
    for (int i = 19; i >= 0; --i) {
        const int owner = i & 3, ri = i >> 2;
        T s = b[ri];
#pragma unroll
        for (int j = i + 1; j < 20; ++j) s -= a[ri][j] * x[j];
        x[i] = __shfl_sync(FULL, s * a[ri][i], owner, 4);
    }
    if (live) {
        T *out = psi + (psi_dir + c) * 20 * (size_t)G + g;
#pragma unroll
        for (int r = 0; r < 5; ++r) out[(size_t)(4 * r + sub) * G] = x[4 * r + sub];
    }
}

// A task: the warp takes its (cell, group) units eight at a time, four lanes per unit.
template <class T>
__device__ __forceinline__ void run_task_p3(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz, size_t psi_dir,
                                            unsigned char *)
{
    const P3Geo<T> *geo = reinterpret_cast<const P3Geo<T> *>(A.geo2);
    const P3Dev<T> *tb = reinterpret_cast<const P3Dev<T> *>(A.p3tab);
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t nu = ncell * (uint32_t)A.G;
    const int slot = lane >> 2, sub = lane & 3;
    for (uint32_t u0 = 0; u0 < nu; u0 += 8) {
        const uint32_t u = u0 + (uint32_t)slot;
        const bool live = u < nu;
        const uint32_t uu = live ? u : u0;  // an idle slot repeats a live unit's cell and discards it
        const uint32_t k = uu / (uint32_t)A.G;
        const int g = (int)(uu - k * (uint32_t)A.G);
        p3_unit4(A, geo, tb, sub, live, __ldg(A.cells + ti.x + k), g, ox, oy, oz, psi_dir);
    }
}
