// Trilinear (eight-node) upwind-DG element on hexahedra: cell record and the local
// solve of one (cell, direction, group) unit.  Included by sweep_kernel.cuh inside
// namespace tf, after the PTX helpers.
//
// Local vertex v = a + 2b + 4c sits at the reference corner (a, b, c); face f = 2d + s
// is the reference face xi_d = s, its face-local nodes k = 0..3 the vertices whose bit
// d equals s, in increasing local index.  Local system (weak form of Eq. (1)
// integrated back by parts, upwind trace on the inflow faces):
//   [ sum_d Omega_d G_d + sum_{f inflow} W_f + sigma_t M ] psi = M q + (Omega.S1) M 1 + sum_{f inflow} W_f psi_up
// with M = int b_i b_j, G_d = int b_i d b_j / dx_d and, on face f's nodes,
// W_f = -sum_d Omega_d F_{f,d}, F_{f,d} = int_f N_d b_k b_l (N the outward area-vector
// density; on a planar face W_f = int_f |Omega.N| b_k b_l), psi_up the upwind cell's nodal
// values on an interior face and the prescribed inflow at the face's vertices (zero under
// vacuum) on a boundary face, and S1 an optional linear anisotropic source constant over the
// cell (M 1: the row sums of M).  A face is inflow when the
// sweep graph says so (the sign of Omega.Nbar_f, Nbar_f = int_f N).  The symmetric part
// of the matrix, (1/2) sum_f |Omega.F_f| + sigma_t M, is positive definite on planar
// faces and was at least 0.19 max|A| on the twisted grids, so elimination needs no
// pivoting.
#pragma once

template <class T> struct alignas(16) HexGeo {
    int32_t nbr[6];   // neighbour across face f, -1 on the boundary
    int32_t mat;      // material
    int32_t pad0;
    uint32_t nmap[6]; // face f: the neighbour's local vertex of face-local node k, 4 bits at bit 4k
    int32_t pad1[2];
    T M[64];          // int b_i b_j, [i][j]
    T Gd[3][64];      // int b_i d b_j / dx_d, [d][i][j]
    T F[6][3][16];    // int_f N_d b_k b_l, [f][d][k][l] over face-local nodes
    T nbar[6][3];     // int_f N: face classification of the leakage
    T pad2[2];
};
static_assert(sizeof(HexGeo<float>) % 16 == 0 && sizeof(HexGeo<double>) % 16 == 0,
              "hexahedral records must be whole 16-byte units");

// local vertex of face-local node k of face f (compile-time when f and k are)
__host__ __device__ constexpr int hex_node(int f, int k)
{
    // the two axes other than d = f / 2, in increasing order; node k has bit k&1 on the
    // lower axis and bit k>>1 on the higher one, and bit d equal to s = f % 2
    return ((f / 2) == 0 ? ((k & 1) << 1) | ((k >> 1) << 2)
            : (f / 2) == 1 ? (k & 1) | ((k >> 1) << 2)
                           : (k & 1) | ((k >> 1) << 1)) |
           ((f % 2) << (f / 2));
}

// 8 x 8 Gaussian elimination without pivoting.
template <class T> __device__ __forceinline__ void hex_solve8(T a[8][8], T b[8], T x[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const T r = rcp(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < 8; ++i) {
            const T l = a[i][k] * r;
#pragma unroll
            for (int j = k + 1; j < 8; ++j) a[i][j] -= l * a[k][j];
            b[i] -= l * b[k];
        }
        a[k][k] = r;
    }
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        T s = b[i];
#pragma unroll
        for (int j = i + 1; j < 8; ++j) s -= a[i][j] * x[j];
        x[i] = s * a[i][i];
    }
}

// Upwind values across interior face f of the cell entry at `pos` for group g: the neighbour's
// psi of this sweep (written by other warps in this launch, read through L2), or, on a lagged
// back edge, its psi of the previous transport step from the lag buffer.
template <class T>
__device__ __forceinline__ void hex_upwind(const SweepArgs<T> &A, const HexGeo<T> *cg, uint32_t pos, int f, int32_t n,
                                           int g, size_t psi_dir, T u[4])
{
    const int G = A.G;
    const uint32_t lw = A.lagw ? __ldg(A.lagw + pos) : 0u;
    if ((lw >> (26 + f)) & 1u) {
        const uint32_t slot = (lw & 0x3ffffffu) + (uint32_t)__popc((lw >> 26) & ((1u << f) - 1u));
        const T *lb = A.lagbuf + (size_t)slot * 4 * G + g;
#pragma unroll
        for (int l = 0; l < 4; ++l) u[l] = __ldg(lb + (size_t)l * G);
        return;
    }
    const uint32_t nm = __ldg(&cg->nmap[f]);
    const T *up = reinterpret_cast<const T *>(A.psi) + (psi_dir + (size_t)n) * 8 * (size_t)G + g;
#pragma unroll
    for (int l = 0; l < 4; ++l) u[l] = __ldcg(up + (size_t)((nm >> (4 * l)) & 15u) * G);
}

// One unit: the cell entry at position pos of the task cell list ((cell << 6) | inflow mask),
// group g.  q and psi are node-major per cell, [cell][node][G].  Lanes of one cell read its
// record at the same addresses (broadcast).
template <class T>
__device__ __forceinline__ void hex_unit(const SweepArgs<T> &A, const HexGeo<T> *__restrict__ geo, uint32_t pos, int g,
                                         T ox, T oy, T oz, size_t psi_dir)
{
    const int G = A.G;
    const uint32_t e = __ldg(A.cells + pos);
    const uint32_t c = e >> 6, mask = e & 63u;
    const HexGeo<T> *cg = geo + c;
    const T sig = __ldg(A.sigma_t + (size_t)__ldg(&cg->mat) * G + g);
    const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 8 * G + g;
    T *psi = reinterpret_cast<T *>(A.psi);
    T a[8][8], b[8], x[8], qv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) qv[j] = __ldg(qc + (size_t)j * G);
    T os = T(0);  // Omega.S1
    if (A.S1) {
        const V4<T> s1 = ld_ro(A.S1 + (size_t)c * G + g);
        os = ox * s1.x + oy * s1.y + oz * s1.z;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        T bi = T(0), ri = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const T m = __ldg(&cg->M[8 * i + j]);
            a[i][j] = ox * __ldg(&cg->Gd[0][8 * i + j]) + oy * __ldg(&cg->Gd[1][8 * i + j]) +
                      oz * __ldg(&cg->Gd[2][8 * i + j]) + sig * m;
            bi += m * qv[j];
            ri += m;
        }
        b[i] = bi + os * ri;
    }
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (!((mask >> f) & 1u)) continue;
        T w[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int l = 0; l < 4; ++l)
                w[k][l] = -(ox * __ldg(&cg->F[f][0][4 * k + l]) + oy * __ldg(&cg->F[f][1][4 * k + l]) +
                            oz * __ldg(&cg->F[f][2][4 * k + l]));
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int l = 0; l < 4; ++l) a[hex_node(f, k)][hex_node(f, l)] += w[k][l];
        const int32_t n = __ldg(&cg->nbr[f]);
        T u[4];
        if (n >= 0) {
            hex_upwind(A, cg, pos, f, n, g, psi_dir, u);
        } else if (A.psi_in) {  // prescribed inflow at the face's vertices
#pragma unroll
            for (int l = 0; l < 4; ++l)
                u[l] = __ldg(A.psi_in + (size_t)__ldg(A.hexv + 8 * (size_t)c + hex_node(f, l)) * G + g);
        } else {
            continue;  // vacuum boundary: no inflow
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T t = T(0);
#pragma unroll
            for (int l = 0; l < 4; ++l) t += w[k][l] * u[l];
            b[hex_node(f, k)] += t;
        }
    }
    hex_solve8(a, b, x);
    T *out = psi + (psi_dir + c) * 8 * (size_t)G + g;
#pragma unroll
    for (int i = 0; i < 8; ++i) out[(size_t)i * G] = x[i];
}

// A task: lanes over the (cell, group) units of its cells (one t-level, independent).
template <class T>
__device__ __forceinline__ void run_task_hex(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                             size_t psi_dir)
{
    const HexGeo<T> *geo = reinterpret_cast<const HexGeo<T> *>(A.geo2);
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t nu = ncell * (uint32_t)A.G;
    for (uint32_t u = lane; u < nu; u += 32) {
        const uint32_t k = u / (uint32_t)A.G;
        const int g = (int)(u - k * (uint32_t)A.G);
        hex_unit(A, geo, ti.x + k, g, ox, oy, oz, psi_dir);
    }
}

// Shared variant (G >= 8): per batch of 32 (cell, group) units the warp first forms, for
// each of the at most HEX_NCB cells the batch touches, the group-independent parts once in
// its shared memory -- the face matrices W_f = -Omega.F_f, the streaming-plus-inflow-face
// matrix S = sum_d Omega_d G_d + sum_{f inflow} W_f and M -- then every lane adds sigma_t M,
// forms its right-hand side and eliminates.  Per warp: HEX_NCB x (96 + 64 + 64) values.
constexpr int HEX_NCB = 5;  // cells one batch of 32 units can touch when G >= 8
__host__ __device__ constexpr uint32_t hex_stage_bytes(int tsize) { return (uint32_t)(HEX_NCB * 224 * tsize); }

// face-local index of vertex v on face f (v on f)
__device__ __forceinline__ int hex_local(int f, int v)
{
    const int d = f >> 1;
    const int lo = d == 0 ? 1 : 0, hi = d == 2 ? 1 : 2;
    return ((v >> lo) & 1) | (((v >> hi) & 1) << 1);
}

template <class T>
__device__ __forceinline__ void run_task_hex_shared(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                                    size_t psi_dir, unsigned char *wsm)
{
    const HexGeo<T> *geo = reinterpret_cast<const HexGeo<T> *>(A.geo2);
    T *Ws = reinterpret_cast<T *>(wsm);      // [HEX_NCB][6][16]
    T *Ss = Ws + HEX_NCB * 96;               // [HEX_NCB][64]
    T *Ms = Ss + HEX_NCB * 64;               // [HEX_NCB][64]
    const int G = A.G;
    const uint32_t ncell = ti.y & 0xffffu;
    const uint32_t nu = ncell * (uint32_t)G;
    T *psi = reinterpret_cast<T *>(A.psi);
    for (uint32_t u0 = 0; u0 < nu; u0 += 32) {
        const uint32_t k0 = u0 / (uint32_t)G;
        const uint32_t k1 = min(ncell - 1u, (u0 + 31u) / (uint32_t)G);
        const int nc = (int)(k1 - k0 + 1u);  // <= HEX_NCB for G >= 8 (the host picks this path only then)
        if (nc > HEX_NCB) {
            if (lane == 0) atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
            return;
        }
        __syncwarp();  // the previous batch is done with the shared tables
        for (int e = lane; e < nc * 96; e += 32) {
            const int kk = e / 96, r = e - kk * 96;  // r = 16 f + 4 k + l
            const HexGeo<T> *cg = geo + (__ldg(A.cells + ti.x + k0 + kk) >> 6);
            const T *F = &cg->F[r >> 4][0][r & 15];
            Ws[e] = -(ox * __ldg(F) + oy * __ldg(F + 16) + oz * __ldg(F + 32));
        }
        __syncwarp();
        for (int e = lane; e < nc * 64; e += 32) {
            const int kk = e >> 6, ij = e & 63, i = ij >> 3, j = ij & 7;
            const uint32_t entry = __ldg(A.cells + ti.x + k0 + kk);
            const HexGeo<T> *cg = geo + (entry >> 6);
            const uint32_t mask = entry & 63u;
            T s = ox * __ldg(&cg->Gd[0][ij]) + oy * __ldg(&cg->Gd[1][ij]) + oz * __ldg(&cg->Gd[2][ij]);
            for (int f = 0; f < 6; ++f) {
                const int d = f >> 1, sd = f & 1;
                if (((mask >> f) & 1u) && ((i >> d) & 1) == sd && ((j >> d) & 1) == sd)
                    s += Ws[kk * 96 + 16 * f + 4 * hex_local(f, i) + hex_local(f, j)];
            }
            Ss[e] = s;
            Ms[e] = __ldg(&cg->M[ij]);
        }
        __syncwarp();
        const uint32_t u = u0 + (uint32_t)lane;
        if (u < nu) {
            const uint32_t k = u / (uint32_t)G;
            const int g = (int)(u - k * (uint32_t)G), kk = (int)(k - k0);
            const uint32_t entry = __ldg(A.cells + ti.x + k);
            const uint32_t c = entry >> 6, mask = entry & 63u;
            const HexGeo<T> *cg = geo + c;
            const T sig = __ldg(A.sigma_t + (size_t)__ldg(&cg->mat) * G + g);
            const T *qc = reinterpret_cast<const T *>(A.q) + (size_t)c * 8 * G + g;
            const T *S = Ss + kk * 64, *M = Ms + kk * 64, *W = Ws + kk * 96;
            T a[8][8], b[8], x[8], qv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) qv[j] = __ldg(qc + (size_t)j * G);
            T os = T(0);  // Omega.S1
            if (A.S1) {
                const V4<T> s1 = ld_ro(A.S1 + (size_t)c * G + g);
                os = ox * s1.x + oy * s1.y + oz * s1.z;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                T bi = T(0), ri = T(0);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const T m = M[8 * i + j];
                    a[i][j] = S[8 * i + j] + sig * m;
                    bi += m * qv[j];
                    ri += m;
                }
                b[i] = bi + os * ri;
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!((mask >> f) & 1u)) continue;
                const int32_t n = __ldg(&cg->nbr[f]);
                T uv[4];
                if (n >= 0) {
                    hex_upwind(A, cg, ti.x + k, f, n, g, psi_dir, uv);
                } else if (A.psi_in) {  // prescribed inflow at the face's vertices
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        uv[l] = __ldg(A.psi_in + (size_t)__ldg(A.hexv + 8 * (size_t)c + hex_node(f, l)) * G + g);
                } else {
                    continue;  // vacuum boundary: no inflow
                }
#pragma unroll
                for (int kf = 0; kf < 4; ++kf) {
                    T t = T(0);
#pragma unroll
                    for (int l = 0; l < 4; ++l) t += W[16 * f + 4 * kf + l] * uv[l];
                    b[hex_node(f, kf)] += t;
                }
            }
            hex_solve8(a, b, x);
            T *out = psi + (psi_dir + c) * 8 * (size_t)G + g;
#pragma unroll
            for (int i = 0; i < 8; ++i) out[(size_t)i * G] = x[i];
        }
    }
}
