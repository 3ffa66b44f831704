// Third-order (twenty-node) upwind-DG element on tetrahedra: cell record, element tables
// and the local solves of one (cell, direction) for all groups.
// Included by sweep_kernel.cuh inside namespace tf, after the PTX helpers.
//
// Nodes: the four vertices, two per edge (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) (first at
// (lambda_a, lambda_b) = (2/3, 1/3)), the four face centres (face f opposite vertex f);
// cubic Lagrange basis on that lattice.  Local system as for the lower orders:
//   [ W + sigma_t V M ] psi = V M q + sum_{f inflow} |Omega.N_f| F_f psi_up,
//   W = V sum_k w_k C_k + sum_{f inflow} |Omega.N_f| F_f,   w_k = Omega . grad lambda_k,
// with the exact tables of p3_tables.cpp (M, C_k per unit volume, F per unit area on the
// face's ten nodes).  W depends on the cell and the direction only: the warp forms it once
// per cell in shared memory, and each group's unit adds sigma_t V M.  A 20 x 20 system does
// not fit one thread's registers, so four lanes share a unit: lane s of the four holds rows
// 4 r + s (r = 0..4) of the matrix and right-hand side in registers; the four are lanes
// u, u + 8, u + 16, u + 24 of the warp (unit u = 0..7), so that the eight lanes holding row k
// form one quarter of the warp.  The elimination takes two columns per step: the lanes holding
// rows k and k + 1 write them to shared memory (one wavefront per 16-byte store), every lane
// reads its unit's two rows back and reduces row k + 1 by row k itself (Gaussian elimination
// without pivoting: the symmetric part, (1/2) sum_f |Omega.N_f| F_f + sigma_t V M, is
// positive definite); the back substitution runs by columns, each unknown broadcast inside
// the four.  A warp solves eight groups of one cell at a time (a pass); the next pass's source
// values are copied into shared memory while the current pass computes.
#pragma once

template <class T> struct alignas(16) P3Geo {
    int32_t nbr[4];              // neighbour across face f, -1 on the boundary
    T gl[12];                    // grad lambda_k, k = 0..3: (x, y, z)
    T nrm[12];                   // area-weighted outward normal N_f of face f
    T vol;                       // V
    int32_t mat;
    unsigned long long fmap[4];  // face f, face node r (0..9): the neighbour's local node, 5 bits at bit 5 r
};

// Element tables as the kernel holds them in shared memory (copied once per CTA).
template <class T> struct alignas(16) P3Dev {
    T M[400];          // int phi_i phi_j / V, row-major
    T C[4][400];       // int phi_i d phi_j / d lambda_k / V
    T FA[4][400];      // F of face f placed in the 20 x 20 matrix (zero off the face's nodes)
    T FU[4][20][12];   // [f][i][c]: F(r, c) for the row i = fn[f][r] of the face, zero elsewhere (c >= 10: 0)
};
static_assert(sizeof(P3Dev<float>) % 16 == 0 && sizeof(P3Dev<double>) % 16 == 0, "tables are copied in 16 B pieces");

// per-warp shared memory of the third-order kernel: the cell's W and two pivot-row buffers of
// eight units (row and right-hand side; a stride of 28 values puts the eight units' 16-byte
// pieces in distinct banks)
constexpr int P3_PSTRIDE = 28;
constexpr int P3_PSTRIDE2 = 60;  // two pivot rows per unit (at 0 and 28); 60 keeps the units' pieces in distinct banks
// and two buffers of the source values of a pass (20 nodes x 8 groups), filled one pass ahead
template <class T> constexpr uint32_t p3_warp_bytes() { return (uint32_t)((400 + 2 * 8 * P3_PSTRIDE2 + 2 * 160) * sizeof(T)); }

// one value copied asynchronously into shared memory (through L1: the source is read-only here)
template <class T> __device__ __forceinline__ void cp_async_elem(T *dst, const T *src)
{
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

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


// Copies the element tables into the CTA's shared memory (all threads; the caller synchronises).
template <class T> __device__ __forceinline__ void p3_stage_tables(const void *src, unsigned char *dst)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(P3Dev<T>) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

// four consecutive values of a row in shared memory (16-byte aligned)
template <class T> struct P3Vec;
template <> struct P3Vec<float> {
    float v[4];
    __device__ __forceinline__ void load(const float *p)
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    __device__ __forceinline__ void store(float *p) const { *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct P3Vec<double> {
    double v[4];
    __device__ __forceinline__ void load(const double *p)
    {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    __device__ __forceinline__ void store(double *p) const
    {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

// A task: per cell, W in shared memory, then the cell's groups eight at a time, four lanes per
// unit.  tb: the element tables in shared memory; wsm: this warp's region (p3_warp_bytes).
template <class T>
__device__ __forceinline__ void run_task_p3(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz, size_t psi_dir,
                                            unsigned char *wsm, const P3Dev<T> *tb)
{
    const unsigned FULL = 0xffffffffu;
    const P3Geo<T> *geo = reinterpret_cast<const P3Geo<T> *>(A.geo2);
    T *Wc = reinterpret_cast<T *>(wsm);  // [20][20]
    T *piv = Wc + 400;                   // [2][8][P3_PSTRIDE2]: two pivot rows (20) and right-hand sides (at 20) per unit
    T *qbuf = piv + 2 * 8 * P3_PSTRIDE2;  // [2][20][8]: the source values of a pass, by node and unit
    const int G = A.G;
    const uint32_t ncell = ti.y & 0xffffu;
    const int slot = lane & 7, sub = lane >> 3;
    T *psi = reinterpret_cast<T *>(A.psi);
    const T *qg = reinterpret_cast<const T *>(A.q);
    // pass p of the task = (cell p / npass, groups 8 (p % npass) ...); its source values are copied
    // into qbuf[p & 1] while pass p - 1 computes
    const uint32_t npass = ((uint32_t)G + 7u) / 8u, n_pass = ncell * npass;
    auto issue_q = [&](uint32_t pp) {
        const uint32_t kq = pp / npass;
        const int gq = (int)(pp - kq * npass) * 8;
        const T *qc = qg + (size_t)(__ldg(A.cells + ti.x + kq) >> 4) * 20 * G;
        T *dst = qbuf + (pp & 1u) * 160;
        for (int t = lane; t < 160; t += 32) {
            const int j = t >> 3, u = t & 7;
            cp_async_elem(dst + t, qc + (size_t)j * G + (gq + u < G ? gq + u : gq));
        }
        cp_async_commit();
    };
    issue_q(0);
    uint32_t pass = 0;
    for (uint32_t kc = 0; kc < ncell; ++kc) {
        const uint32_t e = __ldg(A.cells + ti.x + kc);
        const uint32_t c = e >> 4, mask = e & 15u;
        const P3Geo<T> *cg = geo + c;
        const T V = __ldg(&cg->vol);
        __syncwarp();  // the previous cell's units are done with Wc
        {
            T wv[4], sf[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                wv[k] = V * (ox * __ldg(&cg->gl[3 * k]) + oy * __ldg(&cg->gl[3 * k + 1]) + oz * __ldg(&cg->gl[3 * k + 2]));
                const T sn = ox * __ldg(&cg->nrm[3 * k]) + oy * __ldg(&cg->nrm[3 * k + 1]) + oz * __ldg(&cg->nrm[3 * k + 2]);
                sf[k] = ((mask >> k) & 1u) ? fabs(sn) : T(0);
            }
            for (int q4 = lane; q4 < 100; q4 += 32) {
                P3Vec<T> out, t;
#pragma unroll
                for (int l = 0; l < 4; ++l) out.v[l] = T(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    t.load(&tb->C[k][4 * q4]);
#pragma unroll
                    for (int l = 0; l < 4; ++l) out.v[l] += wv[k] * t.v[l];
                    t.load(&tb->FA[k][4 * q4]);
#pragma unroll
                    for (int l = 0; l < 4; ++l) out.v[l] += sf[k] * t.v[l];
                }
                out.store(Wc + 4 * q4);
            }
        }
        __syncwarp();
        const int32_t mat = __ldg(&cg->mat);
        for (int g0 = 0; g0 < G; g0 += 8) {
            const bool live = g0 + slot < G;
            const int g = live ? g0 + slot : g0;  // an idle slot repeats a live group and discards it
            const T sv = V * __ldg(A.sigma_t + (size_t)mat * G + g);
            // this pass's source values arrived; every lane is done with the buffer refilled next
            cp_async_wait<0>();
            __syncwarp();
            if (pass + 1 < n_pass) issue_q(pass + 1);
            const T *qs = qbuf + (pass & 1u) * 160 + slot;
            ++pass;
            // upwind faces first: b = sum_f s_f F_f psi_up on the face's rows (one loop body for the four faces)
            T b[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) b[r] = T(0);
#pragma unroll 1
            for (int f = 0; f < 4; ++f) {
                const int32_t n = __ldg(&cg->nbr[f]);
                if (!((mask >> f) & 1u) || n < 0) continue;  // vacuum boundary: no inflow
                const T s_f = fabs(ox * __ldg(&cg->nrm[3 * f]) + oy * __ldg(&cg->nrm[3 * f + 1]) + oz * __ldg(&cg->nrm[3 * f + 2]));
                const unsigned long long fm = __ldg(&cg->fmap[f]);
                const T *un = psi + (psi_dir + (size_t)n) * 20 * (size_t)G + g;
                T up[12];
#pragma unroll
                for (int kk = 0; kk < 10; ++kk) up[kk] = __ldcg(un + (size_t)((uint32_t)(fm >> (5 * kk)) & 31u) * G);
                up[10] = up[11] = T(0);
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const T *fu = &tb->FU[f][4 * r + sub][0];
                    T t = T(0);
#pragma unroll
                    for (int c4 = 0; c4 < 3; ++c4) {
                        P3Vec<T> v;
                        v.load(fu + 4 * c4);
#pragma unroll
                        for (int l = 0; l < 4; ++l) t += v.v[l] * up[4 * c4 + l];
                    }
                    b[r] += s_f * t;
                }
            }
            __syncwarp();  // keeps the loads below from being hoisted into the face loop (register pressure)
            // A = W + sigma_t V M and b = V M q in one pass over the lane's rows of W and M
            T a[5][20];
            {
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const T *wr = Wc + 20 * (4 * r + sub);
                    const T *mr = &tb->M[20 * (4 * r + sub)];
                    T bi = T(0);
#pragma unroll
                    for (int j4 = 0; j4 < 5; ++j4) {
                        P3Vec<T> w, m;
                        w.load(wr + 4 * j4);
                        m.load(mr + 4 * j4);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            a[r][4 * j4 + t] = w.v[t] + sv * m.v[t];
                            bi += m.v[t] * qs[8 * (4 * j4 + t)];
                        }
                    }
                    b[r] += V * bi;
                }
            }
            // elimination two columns at a time: rows k and k + 1 (k even) live in lanes (k & 3) and
            // (k & 3) + 1 of the four, both in register row k >> 2.  Both owners write their row (row
            // k + 1 not yet reduced by row k) to the pivot buffer; every lane then reduces row k + 1
            // by row k itself and applies the two pivot rows in the order of single steps.
#pragma unroll
            for (int k = 0; k < 20; k += 2) {
                const int o0 = k & 3, rk = k >> 2, j0 = k & ~3;
                T *pr = piv + ((k >> 1) & 1) * 8 * P3_PSTRIDE2 + slot * P3_PSTRIDE2;
                if (sub == o0 || sub == o0 + 1) {
                    T *dst = pr + (sub == o0 ? 0 : P3_PSTRIDE);
#pragma unroll
                    for (int jj = j0; jj < 20; jj += 4) {
                        P3Vec<T> v;
#pragma unroll
                        for (int l = 0; l < 4; ++l) v.v[l] = a[rk][jj + l];
                        v.store(dst + jj);
                    }
                    dst[20] = b[rk];
                }
                __syncwarp();
                // the piece of both rows holding columns k and k + 1
                P3Vec<T> v0, v1;
                v0.load(pr + j0);
                v1.load(pr + P3_PSTRIDE + j0);
                const T rp0 = rcp(v0.v[k - j0]);
                const T m = v1.v[k - j0] * rp0;                        // row k + 1's multiplier of row k
                const T rp1 = rcp(v1.v[k + 1 - j0] - m * v0.v[k + 1 - j0]);
                const T pb0 = pr[20], pb1 = pr[P3_PSTRIDE + 20] - m * pb0;
                T l0[5], l1[5];
                bool u0[5], u1[5];  // this lane's row is below k / below k + 1
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    u0[r] = 4 * r + 3 > k && (4 * r > k || 4 * r + sub > k);
                    u1[r] = 4 * r + 3 > k + 1 && (4 * r > k + 1 || 4 * r + sub > k + 1);
                    l0[r] = a[r][k] * rp0;
                    // column k + 1 after the reduction by row k, then its multiplier of row k + 1
                    const T ak1 = a[r][k + 1] - l0[r] * v0.v[k + 1 - j0];
                    l1[r] = ak1 * rp1;
                }
                if (sub == o0) a[rk][k] = rp0;  // the owners keep the reciprocals for the back substitution
#pragma unroll
                for (int jj = j0; jj < 20; jj += 4) {
                    if (jj > j0) {
                        v0.load(pr + jj);
                        v1.load(pr + P3_PSTRIDE + jj);
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (jj + t <= k) continue;
                        const T w1 = v1.v[t] - m * v0.v[t];  // row k + 1 reduced by row k
#pragma unroll
                        for (int r = 0; r < 5; ++r) {
                            if (4 * r + 3 <= k) continue;  // rows of this slot are all at or above k
                            if (u0[r]) a[r][jj + t] -= l0[r] * v0.v[t];
                            if (jj + t > k + 1 && u1[r]) a[r][jj + t] -= l1[r] * w1;
                        }
                    }
                }
                if (sub == o0 + 1) a[rk][k + 1] = rp1;
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    if (4 * r + 3 <= k) continue;
                    if (u0[r]) b[r] -= l0[r] * pb0;
                    if (u1[r]) b[r] -= l1[r] * pb1;
                }
            }
            // back substitution by columns: x_i from its owner, then removed from the rows above
#pragma unroll
            for (int i = 19; i >= 0; --i) {
                const int owner = i & 3, ri = i >> 2;
                const T xi = __shfl_sync(FULL, b[ri] * a[ri][i], 8 * owner + slot);
                if (sub == owner) b[ri] = xi;
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    if (4 * r >= i) continue;                          // no row of this slot is above i
                    if (4 * r + 3 >= i && 4 * r + sub >= i) continue;  // this lane's row is not above i
                    b[r] -= a[r][i] * xi;
                }
            }
            if (live) {
                T *out = psi + (psi_dir + c) * 20 * (size_t)G + g;
#pragma unroll
                for (int r = 0; r < 5; ++r) out[(size_t)(4 * r + sub) * G] = b[r];
            }
        }
    }
}

