// Device types, PTX helpers and the persistent sweep kernel (sm_103a).
// Included once, by sweep.cu, inside namespace tf.
#pragma once

// ============================================================== device types
struct alignas(32) double4a {
    double x, y, z, w;
};
template <class T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4a; };
template <class T> using V4 = typename Vec4<T>::type;

// Per-cell geometry in the sweep precision, with the cell's four nodes in
// ascending global-vertex order ("sorted" order; face j is the face opposite
// sorted node j).  In that order the three nodes of a shared face appear in
// the same relative order in both cells, so the upwind trace on a face is the
// upwind cell's nodal vector with one component (the node opposite the face)
// deleted.  g*: (V/4) d b_j / d{x,y,z} (the f_i df_j/dx det J integrals,
// identical for every row i); n*: area-weighted outward normal of face j;
// mv = V/20 (mass matrix scale); code: bits 2j..2j+1 = the neighbour's sorted
// index of the node opposite the shared face j, bits 8+2j..9+2j = the caller's
// local index of sorted node j.
template <class T> struct alignas(16) CellGeo {
    T gx[4], gy[4], gz[4];
    T nx[4], ny[4], nz[4];
    int32_t nbr[4];  // 16-byte aligned: read as one int4 ahead of the record
    T mv;
    int32_t mat;
    uint32_t code;
};
static_assert(sizeof(CellGeo<float>) == 128, "float cell record must be one 128-byte line");
static_assert(sizeof(CellGeo<double>) % 16 == 0, "double cell record must be 16-byte aligned");
static_assert(offsetof(CellGeo<float>, nbr) % 16 == 0 && offsetof(CellGeo<double>, nbr) % 16 == 0,
              "neighbour list must be 16-byte aligned");

// Queue control block.  head/tail live on their own 128-byte lines.
struct Ctrl {
    unsigned long long head;  // next ticket to claim
    unsigned long long pad0[15];
    unsigned long long tail;  // next slot to fill
    unsigned long long pad1[15];
    unsigned long long complete;  // tasks finished in this launch (releases done)
    unsigned long long pad2[15];
    unsigned int epoch;       // tag of the slots filled in the current launch
    int error;                // first device error (TF_ERR_*), 0 if none
    unsigned long long tasks_done;
    unsigned long long polls;
    unsigned long long wait_ns;
    unsigned long long busy_ns;
    unsigned long long t_first;  // earliest warp start (globaltimer)
    unsigned long long t_last;   // latest warp end
    unsigned long long depth_sum;
    unsigned long long pops;
    unsigned long long data_wait_cycles;  // summed over warps: SM cycles waiting for staged rows (bulk copies)
    unsigned long long residual_bits;  // max residual as ordered bits of a non-negative double
    unsigned long long balance_bits;   // max over groups of the relative balance residual (same encoding)
    unsigned long long kernel_ns;      // summed over chunks
    int next_group;                    // next direction group to admit
};

// ============================================================== PTX helpers
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acq_rel(int *p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ float4 ld_ro(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ double4a ld_ro(const double4a *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
// loads of psi written by other warps in the same launch: through L2, never a stale L1 line
__device__ __forceinline__ float4 ld_l2(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ double4a ld_l2(const double4a *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
// streaming loads of the psi store in the phi reduction (read once, evict first)
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ double4a ld_stream(const double4a *p)
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p)), b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st_psi(float4 *p, float4 v) { *p = v; }
__device__ __forceinline__ void st_psi(double4a *p, double4a v)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
}

template <class T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x)
{
    float r;  // one MUFU reciprocal (max error about 1 ulp); the pivots are positive and normal
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ double rcp<double>(double x) { return __drcp_rn(x); }

template <class V> __device__ __forceinline__ auto comp(const V &v, int k) -> decltype(v.x)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// select r[k] for a runtime k in 0..3 without indexing a local array
template <class T> __device__ __forceinline__ T pick4(const T (&r)[4], uint32_t k)
{
    return k == 0u ? r[0] : (k == 1u ? r[1] : (k == 2u ? r[2] : r[3]));
}

// o[perm(j)] = r[j] for the permutation stored in code bits 8+2j..9+2j, by selects
template <class T> __device__ __forceinline__ void scatter4(const T (&r)[4], uint32_t code, T (&o)[4])
{
    const uint32_t p0 = (code >> 8) & 3u, p1 = (code >> 10) & 3u, p2 = (code >> 12) & 3u;
#pragma unroll
    for (uint32_t u = 0; u < 4; ++u) o[u] = p0 == u ? r[0] : (p1 == u ? r[1] : (p2 == u ? r[2] : r[3]));
}

// ============================================================== sweep kernel
template <class T> struct SweepArgs {
    const CellGeo<T> *geo;
    const uint32_t *cells;      // (cell << 4) | inflow mask; hexahedra: (cell << 6) | mask
    const uint4 *task;          // {cell_begin, ncell | dir << 16, down_begin, ndown}
    const uint32_t *down;       // downwind task ids
    int *counters;              // dependency counters
    unsigned long long *slots;  // ready queue, (epoch << 32) | task
    Ctrl *ctrl;
    const V4<T> *q;             // [C][G] angular source per steradian (nodal)
    V4<T> *psi;                 // [Dc][C][G]
    const T *sigma_t;           // [M][G]
    const V4<T> *omega;         // [D] (x, y, z, w)
    const V4<T> *S1;            // [C][G] or NULL
    const T *psi_in;            // [nv][G] or NULL
    const int4 *tets;           // [C] (only with psi_in)
    const int32_t *hexv;        // hexahedra: [C][8] global vertices (only with psi_in)
    // hexahedra with lagged back edges (else NULL): per cell entry (lag mask << 26) | first slot,
    // and per slot the upwind values of the previous transport step, [slot][face-local node][G]
    const uint32_t *lagw;
    const T *lagbuf;
    int64_t C;
    int32_t G;
    int32_t dir_begin;          // first direction of the chunk
    uint32_t task_begin, task_end;
    unsigned long long n_tasks;  // tasks in the chunk
    unsigned long long wait_limit_ns;
    int32_t max_cells;           // largest task (cells)
    uint32_t warp_smem;          // dynamic shared memory per warp (staged path)
    // admission of direction groups (octants): the seeds of group g + window are
    // released when group g is half done
    const int32_t *dir_group;    // [D] group index of each direction within its chunk
    int32_t *group_rem;          // [n_groups] tasks not yet finished (this launch)
    const int32_t *group_admit;  // [n_groups] remaining count that admits the next group
    const uint32_t *gseed;       // [n_groups + 1] seed ranges (offsets into seeds)
    const uint32_t *seeds;
    int32_t n_groups, window;
    int32_t lpc_shift, ppl;      // paired path: log2 lanes per cell, group pairs per lane
    int32_t stages;              // paired path: buffers in the ring of staged copies (2 or 3)
    int32_t mode;                // kernel variant of this problem (batched launches dispatch on it)
    const void *geo2;            // second-order element: P2Geo<T> [C] cell records (modes 5, 6); P3Geo<T> (7); HexGeo<T> (8)
    int32_t keep_max;            // ready tasks a warp keeps and runs next (1..4)
    int32_t intra;               // 1: a task's cells may depend on each other (spatial patches)
    const uint8_t *aux;          // patches, staged variants: per cell entry, its in-task upwind handoffs
    const int32_t *blevel;       // [tasks] longest chain of downwind tasks below each task (global ids), or NULL

    const void *p3tab;           // third-order element: P3Dev<T> tables (mode 7)
};

// Solve one 4x4 system by Gaussian elimination without pivoting: the
// symmetric part of the upwind-DG matrix, (1/2) sum_f |Omega.N_f| M_f +
// sigma_t M, is positive definite, so every pivot is positive.
template <class T> __device__ __forceinline__ void solve4(T a[4][4], T b[4], T x[4])
{
    const T r0 = rcp(a[0][0]);
    const T l10 = a[1][0] * r0, l20 = a[2][0] * r0, l30 = a[3][0] * r0;
    const T a11 = a[1][1] - l10 * a[0][1], a12 = a[1][2] - l10 * a[0][2], a13 = a[1][3] - l10 * a[0][3];
    const T a21 = a[2][1] - l20 * a[0][1], a22 = a[2][2] - l20 * a[0][2], a23 = a[2][3] - l20 * a[0][3];
    const T a31 = a[3][1] - l30 * a[0][1], a32 = a[3][2] - l30 * a[0][2], a33 = a[3][3] - l30 * a[0][3];
    const T b1 = b[1] - l10 * b[0], b2 = b[2] - l20 * b[0], b3 = b[3] - l30 * b[0];
    const T r1 = rcp(a11);
    const T l21 = a21 * r1, l31 = a31 * r1;
    const T c22 = a22 - l21 * a12, c23 = a23 - l21 * a13, c32 = a32 - l31 * a12, c33 = a33 - l31 * a13;
    const T d2 = b2 - l21 * b1, d3 = b3 - l31 * b1;
    const T r2 = rcp(c22);
    const T l32 = c32 * r2;
    const T e33 = c33 - l32 * c23;
    const T e3 = d3 - l32 * d2;
    x[3] = e3 * rcp(e33);
    x[2] = (d2 - c23 * x[3]) * r2;
    x[1] = (b1 - a12 * x[2] - a13 * x[3]) * r1;
    x[0] = (b[0] - a[0][1] * x[1] - a[0][2] * x[2] - a[0][3] * x[3]) * r0;
}

// Group-independent part of one cell's local system for direction Omega, in
// sorted node order, plus the row pointers of its per-group data.
//   A_ij = (V/4) Omega.grad b_j + sum_{f inflow, i,j != f} (|s_f|/12)(1 + delta_ij) + sigma (V/20)(1 + delta_ij)
// With t_f = |s_f|/12 on inflow faces and T = sum_f t_f the face part is
// T - t_i - t_j off the diagonal and 2 (T - t_i) on it.
template <class T> struct Cell {
    T P[4];   // (V/4) Omega.grad b_j
    T t[4];   // |Omega.N_f| / 12 on inflow faces, 0 otherwise
    T tt;     // sum_f t_f
    T mv;     // V/20
    uint32_t c, mask, code;
    int32_t nbr[4];
    const T *sig;         // sigma_t row of the cell's material
};

template <class T>
__device__ __forceinline__ void cell_setup(const SweepArgs<T> &A, uint32_t entry, T ox, T oy, T oz, Cell<T> &s)
{
    s.c = entry >> 4;
    s.mask = entry & 15u;
    union {
        CellGeo<T> g;
        uint4 u[sizeof(CellGeo<T>) / 16];
    } U;
    const uint4 *src = reinterpret_cast<const uint4 *>(A.geo + s.c);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(CellGeo<T>) / 16); ++k) U.u[k] = __ldg(src + k);
    const CellGeo<T> &g = U.g;
    s.tt = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) s.P[j] = ox * g.gx[j] + oy * g.gy[j] + oz * g.gz[j];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T sf = ox * g.nx[f] + oy * g.ny[f] + oz * g.nz[f];
        s.t[f] = ((s.mask >> f) & 1u) ? fabs(sf) * T(1.0 / 12.0) : T(0);
        s.tt += s.t[f];
    }
    s.mv = g.mv;
    s.code = g.code;
    s.sig = A.sigma_t + (size_t)g.mat * A.G;
#pragma unroll
    for (int f = 0; f < 4; ++f) s.nbr[f] = g.nbr[f];
}

// Inputs of one (cell, direction, group) unit, loaded before any arithmetic so
// that the loads of several units are in flight together.
template <class T> struct UnitIn {
    V4<T> q;
    V4<T> u[4];  // upwind cell's psi across face f (zero if not an interior inflow face)
    T sig;
};

template <class T>
__device__ __forceinline__ void unit_load(const SweepArgs<T> &A, const Cell<T> &s, int g, size_t psi_dir,
                                          UnitIn<T> &in)
{
    const int G = A.G;
    in.sig = __ldg(s.sig + g);
    in.q = ld_ro(A.q + (size_t)s.c * G + g);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (((s.mask >> f) & 1u) && s.nbr[f] >= 0) {
            in.u[f] = ld_l2(A.psi + (psi_dir + (size_t)s.nbr[f]) * G + g);
        } else {
            in.u[f].x = in.u[f].y = in.u[f].z = in.u[f].w = T(0);
        }
    }
}

// Assemble and solve one unit from its loaded inputs; store psi (sorted order).
template <class T>
__device__ __forceinline__ void unit_solve(const SweepArgs<T> &A, const Cell<T> &s, int g, size_t psi_dir,
                                           const UnitIn<T> &in, T ox, T oy, T oz)
{
    const int G = A.G;
    const T sv = in.sig * s.mv;
    const T qs = (in.q.x + in.q.y) + (in.q.z + in.q.w);
    T b[4] = {s.mv * (in.q.x + qs), s.mv * (in.q.y + qs), s.mv * (in.q.z + qs), s.mv * (in.q.w + qs)};
    if (A.S1) {
        const V4<T> s1 = ld_ro(A.S1 + (size_t)s.c * G + g);
        const T os = T(5) * s.mv * (ox * s1.x + oy * s1.y + oz * s1.z);  // (V/4) Omega.S1
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] += os;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!((s.mask >> f) & 1u)) continue;
        T v0, v1, v2;  // upwind trace at the face's nodes, ascending global id
        if (s.nbr[f] >= 0) {
            const uint32_t fn = (s.code >> (2 * f)) & 3u;  // upwind node opposite the face
            const V4<T> &u = in.u[f];
            v0 = fn == 0u ? u.y : u.x;
            v1 = fn <= 1u ? u.z : u.y;
            v2 = fn <= 2u ? u.w : u.z;
        } else if (A.psi_in) {
            const int4 tv = __ldg(A.tets + s.c);
            const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
            const int i0 = f == 0 ? 1 : 0, i1 = f <= 1 ? 2 : 1, i2 = f <= 2 ? 3 : 2;
            v0 = __ldg(A.psi_in + (size_t)vi[i0] * G + g);
            v1 = __ldg(A.psi_in + (size_t)vi[i1] * G + g);
            v2 = __ldg(A.psi_in + (size_t)vi[i2] * G + g);
        } else {
            continue;  // vacuum: no inflow
        }
        const T U = v0 + v1 + v2;
        // the face's nodes in sorted order are {0..3} \ {f}, ascending
        b[f == 0 ? 1 : 0] += s.t[f] * (v0 + U);
        b[f <= 1 ? 2 : 1] += s.t[f] * (v1 + U);
        b[f <= 2 ? 3 : 2] += s.t[f] * (v2 + U);
    }
    T a[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            a[i][j] = s.P[j] + (i == j ? T(2) * (s.tt - s.t[i] + sv) : (s.tt - s.t[i] - s.t[j]) + sv);
    T x[4];
    solve4(a, b, x);
    V4<T> out;
    out.x = x[0];
    out.y = x[1];
    out.z = x[2];
    out.w = x[3];
    st_psi(A.psi + (psi_dir + (size_t)s.c) * G + g, out);
}

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// One task when every cell's groups fill whole warps (G a multiple of 32 and
// at most 64 cells per task): lane l solves groups l, l+32, ... of each cell,
// two units' loads in flight at once; the next cell's record and source rows
// are prefetched into L1 while the current cell is solved.
template <class T>
__device__ __forceinline__ void run_task_wide(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                              size_t psi_dir)
{
    const uint32_t ncell = ti.y & 0xffffu;
    const unsigned FULL = 0xffffffffu;
    const uint32_t e_lo = lane < (int)ncell ? __ldg(A.cells + ti.x + lane) : 0u;
    const uint32_t e_hi = lane + 32 < (int)ncell ? __ldg(A.cells + ti.x + 32 + lane) : 0u;
    const int G = A.G;
    const size_t row_bytes = (size_t)G * sizeof(V4<T>);
    for (uint32_t k = 0; k < ncell; ++k) {
        const uint32_t e = __shfl_sync(FULL, k < 32 ? e_lo : e_hi, k & 31);
        if (k + 1 < ncell) {
            const uint32_t e1 = __shfl_sync(FULL, k + 1 < 32 ? e_lo : e_hi, (k + 1) & 31);
            const uint32_t c1 = e1 >> 4;
            const char *qrow = reinterpret_cast<const char *>(A.q + (size_t)c1 * G);
            for (size_t off = (size_t)lane * 128; off < row_bytes; off += 32 * 128) prefetch_l1(qrow + off);
            if (lane < (int)((sizeof(CellGeo<T>) + 127) / 128))
                prefetch_l1(reinterpret_cast<const char *>(A.geo + c1) + 128 * lane);
        }
        Cell<T> s;
        cell_setup(A, e, ox, oy, oz, s);
        int g = lane;
        for (; g + 32 < G; g += 64) {
            UnitIn<T> in0, in1;
            unit_load(A, s, g, psi_dir, in0);
            unit_load(A, s, g + 32, psi_dir, in1);
            unit_solve(A, s, g, psi_dir, in0, ox, oy, oz);
            unit_solve(A, s, g + 32, psi_dir, in1, ox, oy, oz);
        }
        if (g < G) {
            UnitIn<T> in0;
            unit_load(A, s, g, psi_dir, in0);
            unit_solve(A, s, g, psi_dir, in0, ox, oy, oz);
        }
    }
}

// Any group count and task size: units u = lane, lane + 32, ... over
// (cell k, group g), g fastest; the cell setup is redone when k changes.
template <class T>
__device__ __forceinline__ void run_task_generic(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                                 size_t psi_dir)
{
    const uint32_t ncell = ti.y & 0xffffu;
    int g = lane;
    uint32_t k = 0;
    while (g >= A.G) {
        g -= A.G;
        ++k;
    }
    uint32_t kc = 0xffffffffu;
    Cell<T> s;
    while (k < ncell) {
        if (k != kc) {
            cell_setup(A, __ldg(A.cells + ti.x + k), ox, oy, oz, s);
            kc = k;
        }
        UnitIn<T> in;
        unit_load(A, s, g, psi_dir, in);
        unit_solve(A, s, g, psi_dir, in, ox, oy, oz);
        g += 32;
        while (g >= A.G) {
            g -= A.G;
            ++k;
        }
    }
}

// ------------------------------------------------------------------ TMA staging
// One warp stages, per cell, its geometry record, its source row q[c][0..G)
// and the psi rows of its (at most three) interior inflow neighbours into
// shared memory with bulk asynchronous copies (cp.async.bulk, completion on
// an mbarrier), three cells ahead of the one being solved.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Per-thread asynchronous 16-byte copy global -> shared (through L2, not L1), tracked by the
// thread's commit groups; no proxy change: the copy reads and writes as the thread itself does.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// The entries gg = lane, lane + 32, ... < G of one row (V4<T> each) copied by the lane that reads them.
template <class T, int NPL = 0> __device__ __forceinline__ void copy_row_own(V4<T> *dst, const V4<T> *src, int lane, int G)
{
    if constexpr (NPL > 0) {  // G = 32 NPL: the lane's entries without a loop
#pragma unroll
        for (int k = 0; k < NPL; ++k)
#pragma unroll
            for (int h = 0; h < (int)(sizeof(V4<T>) / 16); ++h)
                cp_async16(reinterpret_cast<char *>(dst + lane + 32 * k) + 16 * h,
                           reinterpret_cast<const char *>(src + lane + 32 * k) + 16 * h);
    } else {
        for (int gg = lane; gg < G; gg += 32) {
#pragma unroll
            for (int h = 0; h < (int)(sizeof(V4<T>) / 16); ++h)
                cp_async16(reinterpret_cast<char *>(dst + gg) + 16 * h, reinterpret_cast<const char *>(src + gg) + 16 * h);
        }
    }
}

// Bounded wait on an mbarrier phase; false (and the error word set) after limit_ns.
// Lane 0 adds the SM cycles it spent in the wait (try_wait may suspend the
// thread inside the first attempt) to *acc, the warp's data-wait counter.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns, int *err,
                                          unsigned long long *acc)
{
    const long long c0 = clock64();
    if (!mbar_try_wait(bar, parity)) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(bar, parity)) {
            if (globaltimer() - t0 > limit_ns) {
                atomicCAS(err, 0, (int)TF_ERR_TIMEOUT);
                return false;
            }
        }
    }
    if ((threadIdx.x & 31) == 0) *acc += (unsigned long long)(clock64() - c0);
    return true;
}

template <class T> struct StageLayout {
    uint32_t row;    // G psi/q entries
    uint32_t stage;  // geometry record + q row + 3 upwind rows
    __device__ __forceinline__ StageLayout(int G)
        : row((uint32_t)G * (uint32_t)sizeof(V4<T>)), stage((uint32_t)sizeof(CellGeo<T>) + 4u * row)
    {
    }
};

// Bytes of shared memory one warp needs for the staged path's NS stages (the mbarriers come on top).
template <class T> inline size_t staged_warp_bytes(int G, int NS = 3)
{
    return (size_t)NS * (sizeof(CellGeo<T>) + 4 * (size_t)G * sizeof(V4<T>));
}

// Packed FP32 pairs: both halves of a 64-bit register hold one group each and
// Blackwell's add/mul/fma.rn.f32x2 operate on both.
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 a, float &x, float &y) { asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ f2 sel2(bool p, f2 a, f2 b)
{
    f2 r;
    r.v = p ? a.v : b.v;
    return r;
}
// -1 / a, halfwise (one MUFU reciprocal each)
__device__ __forceinline__ f2 nrcp2(f2 a)
{
    float x, y;
    upk(a, x, y);
    return pk(rcp<float>(-x), rcp<float>(-y));
}

// Solve every group of one staged cell: lane l takes groups l, l+32, ...
// NPL > 0: exactly NPL groups per lane (G = 32 NPL), unrolled so that the
// independent solves of a lane's groups interleave; NPL = 0: any G.
// fill0 / fill1: when not NULL, shared-memory upwind rows of later cells of the same task
// (spatial patches) that take this cell's solution; each lane writes the entries it solves.
template <class T, int NPL>
__device__ __forceinline__ void solve_staged_cell(const SweepArgs<T> &A, const unsigned char *st_base, uint32_t entry,
                                                  int lane, T ox, T oy, T oz, size_t psi_dir, const StageLayout<T> &L,
                                                  V4<T> *fill0, V4<T> *fill1)
{
    const CellGeo<T> &g = *reinterpret_cast<const CellGeo<T> *>(st_base);
    const V4<T> *qrow = reinterpret_cast<const V4<T> *>(st_base + sizeof(CellGeo<T>));
    const uint32_t c = entry >> 4, mask = entry & 15u;
    T P[4], t[4], tt = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) P[j] = ox * g.gx[j] + oy * g.gy[j] + oz * g.gz[j];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T sf = ox * g.nx[f] + oy * g.ny[f] + oz * g.nz[f];
        t[f] = ((mask >> f) & 1u) ? fabs(sf) * T(1.0 / 12.0) : T(0);
        tt += t[f];
    }
    const T mv = g.mv;
    const uint32_t code = g.code;
    int32_t nb[4];
    const V4<T> *uprow[4];
    uint32_t slot = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        nb[f] = g.nbr[f];
        const bool up = ((mask >> f) & 1u) && nb[f] >= 0;
        uprow[f] = reinterpret_cast<const V4<T> *>(st_base + sizeof(CellGeo<T>) + (1 + slot) * L.row);
        slot += up ? 1u : 0u;
    }
    const T *sig = A.sigma_t + (size_t)g.mat * A.G;
    V4<T> *out = A.psi + (psi_dir + (size_t)c) * A.G;
    // group-independent part of the matrix; the group adds sigma_t (V/20)(1 + delta_ij)
    T Bm[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Bm[i][j] = P[j] + (i == j ? T(2) * (tt - t[i]) : (tt - t[i]) - t[j]);
    auto unit = [&](int gg) {
        const T sv = __ldg(sig + gg) * mv;
        const V4<T> q4 = qrow[gg];
        const T qs = (q4.x + q4.y) + (q4.z + q4.w);
        T b[4] = {mv * (q4.x + qs), mv * (q4.y + qs), mv * (q4.z + qs), mv * (q4.w + qs)};
        if (A.S1) {
            const V4<T> s1 = ld_ro(A.S1 + (size_t)c * A.G + gg);
            const T os = T(5) * mv * (ox * s1.x + oy * s1.y + oz * s1.z);
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] += os;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (!((mask >> f) & 1u)) continue;
            T v0, v1, v2;
            if (nb[f] >= 0) {
                const uint32_t fn = (code >> (2 * f)) & 3u;
                const V4<T> u = uprow[f][gg];
                v0 = fn == 0u ? u.y : u.x;
                v1 = fn <= 1u ? u.z : u.y;
                v2 = fn <= 2u ? u.w : u.z;
            } else if (A.psi_in) {
                const int4 tv = __ldg(A.tets + c);
                const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
                v0 = __ldg(A.psi_in + (size_t)vi[f == 0 ? 1 : 0] * A.G + gg);
                v1 = __ldg(A.psi_in + (size_t)vi[f <= 1 ? 2 : 1] * A.G + gg);
                v2 = __ldg(A.psi_in + (size_t)vi[f <= 2 ? 3 : 2] * A.G + gg);
            } else {
                continue;
            }
            const T U = v0 + v1 + v2;
            b[f == 0 ? 1 : 0] += t[f] * (v0 + U);
            b[f <= 1 ? 2 : 1] += t[f] * (v1 + U);
            b[f <= 2 ? 3 : 2] += t[f] * (v2 + U);
        }
        T a[4][4];
        const T sv2 = T(2) * sv;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a[i][j] = Bm[i][j] + (i == j ? sv2 : sv);
        T x[4];
        solve4(a, b, x);
        V4<T> o;
        o.x = x[0];
        o.y = x[1];
        o.z = x[2];
        o.w = x[3];
        st_psi(out + gg, o);
        if (fill0) fill0[gg] = o;
        if (fill1) fill1[gg] = o;
    };
    if constexpr (NPL == 2 && sizeof(T) == 4) {
        // G = 64, FP32: the lane's two groups (lane, lane + 32) packed into f32x2 pairs,
        // so the right-hand side, the matrix and the elimination take one packed
        // instruction for both (the reciprocals stay one MUFU per half)
        const float4 qa = reinterpret_cast<const float4 *>(qrow)[lane], qb = reinterpret_cast<const float4 *>(qrow)[lane + 32];
        const f2 mvp = pk(mv, mv);
        const f2 sv = pk(__ldg(sig + lane), __ldg(sig + lane + 32)) * mvp;
        const f2 qx = pk(qa.x, qb.x), qy = pk(qa.y, qb.y), qz = pk(qa.z, qb.z), qw = pk(qa.w, qb.w);
        const f2 qs = (qx + qy) + (qz + qw);
        f2 b[4] = {mvp * (qx + qs), mvp * (qy + qs), mvp * (qz + qs), mvp * (qw + qs)};
        if (A.S1) {
            const float4 s0 = __ldg(reinterpret_cast<const float4 *>(A.S1) + (size_t)c * A.G + lane);
            const float4 s1 = __ldg(reinterpret_cast<const float4 *>(A.S1) + (size_t)c * A.G + lane + 32);
            const f2 os = pk(5.f * mv * (ox * s0.x + oy * s0.y + oz * s0.z), 5.f * mv * (ox * s1.x + oy * s1.y + oz * s1.z));
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = b[i] + os;
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (!((mask >> f) & 1u)) continue;
            const int i0 = f == 0 ? 1 : 0, i1 = f <= 1 ? 2 : 1, i2 = f <= 2 ? 3 : 2;
            f2 v0, v1, v2;
            if (nb[f] >= 0) {
                const uint32_t fn = (code >> (2 * f)) & 3u;  // upwind node opposite the face
                const bool s0 = fn == 0u, s1 = fn <= 1u, s2 = fn <= 2u;
                const float4 ua = reinterpret_cast<const float4 *>(uprow[f])[lane];
                const float4 ub = reinterpret_cast<const float4 *>(uprow[f])[lane + 32];
                v0 = pk(s0 ? ua.y : ua.x, s0 ? ub.y : ub.x);
                v1 = pk(s1 ? ua.z : ua.y, s1 ? ub.z : ub.y);
                v2 = pk(s2 ? ua.w : ua.z, s2 ? ub.w : ub.z);
            } else if (A.psi_in) {
                const int4 tv = __ldg(A.tets + c);
                const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
                const float *pi = reinterpret_cast<const float *>(A.psi_in);
                v0 = pk(__ldg(pi + (size_t)vi[i0] * A.G + lane), __ldg(pi + (size_t)vi[i0] * A.G + lane + 32));
                v1 = pk(__ldg(pi + (size_t)vi[i1] * A.G + lane), __ldg(pi + (size_t)vi[i1] * A.G + lane + 32));
                v2 = pk(__ldg(pi + (size_t)vi[i2] * A.G + lane), __ldg(pi + (size_t)vi[i2] * A.G + lane + 32));
            } else {
                continue;  // vacuum
            }
            const f2 tf = pk(t[f], t[f]);
            const f2 Uf = (v0 + v1) + v2;
            b[i0] = fma2(tf, v0 + Uf, b[i0]);
            b[i1] = fma2(tf, v1 + Uf, b[i1]);
            b[i2] = fma2(tf, v2 + Uf, b[i2]);
        }
        const f2 two = pk(2.f, 2.f);
        f2 a[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const f2 w = pk(Bm[i][j], Bm[i][j]);
                a[i][j] = i == j ? fma2(two, sv, w) : w + sv;
            }
        // elimination with n_ik = -a_ik / a_kk, back substitution on y = -x
        const f2 nr0 = nrcp2(a[0][0]);
        const f2 n10 = a[1][0] * nr0, n20 = a[2][0] * nr0, n30 = a[3][0] * nr0;
        const f2 a11 = fma2(n10, a[0][1], a[1][1]), a12 = fma2(n10, a[0][2], a[1][2]), a13 = fma2(n10, a[0][3], a[1][3]);
        const f2 a21 = fma2(n20, a[0][1], a[2][1]), a22 = fma2(n20, a[0][2], a[2][2]), a23 = fma2(n20, a[0][3], a[2][3]);
        const f2 a31 = fma2(n30, a[0][1], a[3][1]), a32 = fma2(n30, a[0][2], a[3][2]), a33 = fma2(n30, a[0][3], a[3][3]);
        const f2 b1 = fma2(n10, b[0], b[1]), b2 = fma2(n20, b[0], b[2]), b3 = fma2(n30, b[0], b[3]);
        const f2 nr1 = nrcp2(a11);
        const f2 n21 = a21 * nr1, n31 = a31 * nr1;
        const f2 c22 = fma2(n21, a12, a22), c23 = fma2(n21, a13, a23), c32 = fma2(n31, a12, a32), c33 = fma2(n31, a13, a33);
        const f2 d2 = fma2(n21, b1, b2), d3 = fma2(n31, b1, b3);
        const f2 nr2 = nrcp2(c22);
        const f2 n32 = c32 * nr2;
        const f2 e33 = fma2(n32, c23, c33), e3 = fma2(n32, d2, d3);
        const f2 y3 = e3 * nrcp2(e33);
        const f2 y2 = fma2(c23, y3, d2) * nr2;
        const f2 y1 = fma2(a13, y3, fma2(a12, y2, b1)) * nr1;
        const f2 y0 = fma2(a[0][3], y3, fma2(a[0][2], y2, fma2(a[0][1], y1, b[0]))) * nr0;
        float x0a, x0b, x1a, x1b, x2a, x2b, x3a, x3b;
        upk(y0, x0a, x0b);
        upk(y1, x1a, x1b);
        upk(y2, x2a, x2b);
        upk(y3, x3a, x3b);
        const float4 oa = make_float4(-x0a, -x1a, -x2a, -x3a), ob = make_float4(-x0b, -x1b, -x2b, -x3b);
        reinterpret_cast<float4 *>(out)[lane] = oa;
        reinterpret_cast<float4 *>(out)[lane + 32] = ob;
        if (fill0) {
            reinterpret_cast<float4 *>(fill0)[lane] = oa;
            reinterpret_cast<float4 *>(fill0)[lane + 32] = ob;
        }
        if (fill1) {
            reinterpret_cast<float4 *>(fill1)[lane] = oa;
            reinterpret_cast<float4 *>(fill1)[lane + 32] = ob;
        }
    } else if constexpr (NPL > 0) {
        // the lane's NPL groups side by side: every face test and trace selection is made
        // once per cell and the independent solves interleave
        T sv[NPL], b[NPL][4];
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const int gg = lane + 32 * k;
            sv[k] = __ldg(sig + gg) * mv;
            const V4<T> q4 = qrow[gg];
            const T qs = (q4.x + q4.y) + (q4.z + q4.w);
            b[k][0] = mv * (q4.x + qs);
            b[k][1] = mv * (q4.y + qs);
            b[k][2] = mv * (q4.z + qs);
            b[k][3] = mv * (q4.w + qs);
        }
        if (A.S1) {
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const V4<T> s1 = ld_ro(A.S1 + (size_t)c * A.G + lane + 32 * k);
                const T os = T(5) * mv * (ox * s1.x + oy * s1.y + oz * s1.z);
#pragma unroll
                for (int i = 0; i < 4; ++i) b[k][i] += os;
            }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (!((mask >> f) & 1u)) continue;
            // the face's nodes in sorted order are {0..3} \ {f}, ascending
            const int i0 = f == 0 ? 1 : 0, i1 = f <= 1 ? 2 : 1, i2 = f <= 2 ? 3 : 2;
            if (nb[f] >= 0) {
                const uint32_t fn = (code >> (2 * f)) & 3u;  // upwind node opposite the face
                const bool s0 = fn == 0u, s1 = fn <= 1u, s2 = fn <= 2u;
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    const V4<T> u = uprow[f][lane + 32 * k];
                    const T v0 = s0 ? u.y : u.x, v1 = s1 ? u.z : u.y, v2 = s2 ? u.w : u.z;
                    const T U = v0 + v1 + v2;
                    b[k][i0] += t[f] * (v0 + U);
                    b[k][i1] += t[f] * (v1 + U);
                    b[k][i2] += t[f] * (v2 + U);
                }
            } else if (A.psi_in) {
                const int4 tv = __ldg(A.tets + c);
                const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    const int gg = lane + 32 * k;
                    const T v0 = __ldg(A.psi_in + (size_t)vi[i0] * A.G + gg);
                    const T v1 = __ldg(A.psi_in + (size_t)vi[i1] * A.G + gg);
                    const T v2 = __ldg(A.psi_in + (size_t)vi[i2] * A.G + gg);
                    const T U = v0 + v1 + v2;
                    b[k][i0] += t[f] * (v0 + U);
                    b[k][i1] += t[f] * (v1 + U);
                    b[k][i2] += t[f] * (v2 + U);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            T a[4][4];
            const T sv2 = T(2) * sv[k];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = Bm[i][j] + (i == j ? sv2 : sv[k]);
            T x[4];
            solve4(a, b[k], x);
            V4<T> o;
            o.x = x[0];
            o.y = x[1];
            o.z = x[2];
            o.w = x[3];
            st_psi(out + lane + 32 * k, o);
            if (fill0) fill0[lane + 32 * k] = o;
            if (fill1) fill1[lane + 32 * k] = o;
        }
    } else {
        for (int gg = lane; gg < A.G; gg += 32) unit(gg);
    }
}

// One task through the staged pipeline.  Stage of cell k = k mod NS holds its
// cell record, its source row and its upwind rows (interior inflow faces in face
// order).  The copies of cell k are issued NS - 1 cells ahead of its solve as
// per-lane asynchronous 16-byte copies (cp.async): each lane copies the entries
// of the rows it will itself read (groups lane, lane + 32, ...), lanes 0.. the
// record that every lane reads; each issue is one commit group per lane, and a
// solve first waits until its cell's group is complete (then the warp syncs, for
// the record).  No copy goes through the bulk-copy unit, so no issue queues behind
// another warp's copies.  Returns false if a wait ran out (error word set).
// Spatial patches (A.intra): an upwind cell may be cell p < k of the same task; the
// host marks each cell entry (A.aux, one byte).  If p was solved before cell k's
// copies are issued (p <= k - NS), each lane copies its own entries of p's row back
// (L2; the lane wrote them itself); otherwise the lanes write the entries of p's
// solution they computed into k's upwind slot as they finish p.
template <class T, int NPL, int NS = 3>
__device__ __forceinline__ bool run_task_staged(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                                size_t psi_dir, unsigned char *wsm, uint64_t *, uint32_t &,
                                                unsigned long long *wacc)
{
    static_assert(NS == 2 || NS == 3, "two or three stages");
    const unsigned FULL = 0xffffffffu;
    const uint32_t ncell = ti.y & 0xffffu;
    const StageLayout<T> L(A.G);
    const uint32_t e_lo = lane < (int)ncell ? __ldg(A.cells + ti.x + lane) : 0u;
    const uint32_t e_hi = lane + 32 < (int)ncell ? __ldg(A.cells + ti.x + 32 + lane) : 0u;
    const bool intra = A.intra != 0;
    const uint32_t a_lo = intra && lane < (int)ncell ? (uint32_t)__ldg(A.aux + ti.x + lane) : 0u;
    const uint32_t a_hi = intra && lane + 32 < (int)ncell ? (uint32_t)__ldg(A.aux + ti.x + 32 + lane) : 0u;
    int4 n_lo = make_int4(-1, -1, -1, -1), n_hi = n_lo;
    if (lane < (int)ncell) n_lo = __ldg(reinterpret_cast<const int4 *>(A.geo[e_lo >> 4].nbr));
    if (lane + 32 < (int)ncell) n_hi = __ldg(reinterpret_cast<const int4 *>(A.geo[e_hi >> 4].nbr));
    constexpr int REC_CHUNKS = (int)(sizeof(CellGeo<T>) / 16);
    auto issue = [&](uint32_t k) {
        const int src = (int)(k & 31u);
        const bool hi = k >= 32u;
        const uint32_t ek = __shfl_sync(FULL, hi ? e_hi : e_lo, src);
        const uint32_t ak = intra ? __shfl_sync(FULL, hi ? a_hi : a_lo, src) : 0u;
        int nb[4];
        nb[0] = __shfl_sync(FULL, hi ? n_hi.x : n_lo.x, src);
        nb[1] = __shfl_sync(FULL, hi ? n_hi.y : n_lo.y, src);
        nb[2] = __shfl_sync(FULL, hi ? n_hi.z : n_lo.z, src);
        nb[3] = __shfl_sync(FULL, hi ? n_hi.w : n_lo.w, src);
        const uint32_t s = k % (uint32_t)NS, mask = ek & 15u, c = ek >> 4;
        unsigned char *st = wsm + s * L.stage;
        if (lane < REC_CHUNKS)
            cp_async16(st + 16 * lane, reinterpret_cast<const char *>(A.geo + c) + 16 * lane);
        copy_row_own<T, NPL>(reinterpret_cast<V4<T> *>(st + sizeof(CellGeo<T>)), A.q + (size_t)c * A.G, lane, A.G);
        uint32_t r = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (!((mask >> f) & 1u) || nb[f] < 0) continue;
            if (!((ak >> r) & 1u))  // not handed over by the lanes: copy this lane's entries of the row
                copy_row_own<T, NPL>(reinterpret_cast<V4<T> *>(st + sizeof(CellGeo<T>) + (1u + r) * L.row),
                                     A.psi + (psi_dir + (size_t)nb[f]) * A.G, lane, A.G);
            ++r;
        }
        cp_async_commit();
    };
    issue(0);
    if (NS == 3) {
        if (ncell > 1)
            issue(1);
        else
            cp_async_commit();
    }
    for (uint32_t k = 0; k < ncell; ++k) {
        const uint32_t s = k % (uint32_t)NS;
        const uint32_t ek = __shfl_sync(FULL, k < 32 ? e_lo : e_hi, k & 31);
        const uint32_t ak = intra ? __shfl_sync(FULL, k < 32 ? a_lo : a_hi, k & 31) : 0u;
        if (k + NS - 1 < ncell)
            issue(k + NS - 1);
        else
            cp_async_commit();  // an empty group keeps NS - 1 groups behind this cell's
        const long long c0 = clock64();
        cp_async_wait<NS - 1>();
        __syncwarp();  // the record, copied by lanes 0.., is read by every lane
        if (lane == 0) *wacc += (unsigned long long)(clock64() - c0);
        // the upwind slots of the next cells (already issued) that take this cell's solution
        V4<T> *fill0 = nullptr, *fill1 = nullptr;
        if (ak & 0x30u)
            fill0 = reinterpret_cast<V4<T> *>(wsm + ((k + 1) % (uint32_t)NS) * L.stage + sizeof(CellGeo<T>) +
                                              ((ak >> 4) & 3u) * L.row);
        if (NS == 3 && (ak & 0xc0u))
            fill1 = reinterpret_cast<V4<T> *>(wsm + ((k + 2) % (uint32_t)NS) * L.stage + sizeof(CellGeo<T>) +
                                              ((ak >> 6) & 3u) * L.row);
        solve_staged_cell<T, NPL>(A, wsm + s * L.stage, ek, lane, ox, oy, oz, psi_dir, L, fill0, fill1);
        __syncwarp();  // every lane has read the stage's record before a later issue overwrites it
    }
    return true;
}

// ------------------------------------------------------------------ packed pairs
// FP32 mode, even G: a lane solves two groups of one cell at once.  Both
// groups' values of a quantity share one 64-bit register and Blackwell's
// packed FP32 instructions (add/sub/mul/fma .f32x2) operate on both halves.
// The source and psi rows are stored pair-interleaved, [cell][G/2][node][2],
// so one 32-byte load yields the four packed nodal values of a group pair.
struct P4 {
    f2 x, y, z, w;  // node 0..3, each packed (group 2p, group 2p+1)
};
__device__ __forceinline__ P4 ld_pair_ro(const float *p)
{
    const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(p)), b = __ldg(reinterpret_cast<const ulonglong2 *>(p) + 1);
    return {{a.x}, {a.y}, {b.x}, {b.y}};
}
__device__ __forceinline__ P4 ld_pair_l2(const float *p)
{
    const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2 *>(p)), b = __ldcg(reinterpret_cast<const ulonglong2 *>(p) + 1);
    return {{a.x}, {a.y}, {b.x}, {b.y}};
}
__device__ __forceinline__ void st_pair(float *p, const P4 &v)
{
    reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(v.x.v, v.y.v);
    reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(v.z.v, v.w.v);
}

// Cell table of the paired path: one 256-byte row per task cell, written once
// per task by the lane that owns the cell (lane-parallel setup) and read by
// every lane that solves one of the cell's group pairs.  W is the
// group-independent matrix part (A = W + sigma (V/20)(1 + delta_ij)), t the
// inflow face weights, mv = V/20, all broadcast into both halves.
struct TabRow {
    f2 W[4][4];
    f2 t[4];
    f2 mv;
    uint32_t c, mask, code;
    int32_t mat;
    int32_t nbr[4];
    uint32_t upmask;  // interior inflow faces (their psi rows are staged, in face order)
    uint32_t pad[13];
};
static_assert(sizeof(TabRow) == 256, "table row must be 256 bytes");

__device__ __forceinline__ void tab_setup(const SweepArgs<float> &A, uint32_t entry, float ox, float oy, float oz,
                                          TabRow &r)
{
    const uint32_t c = entry >> 4, mask = entry & 15u;
    union {
        CellGeo<float> g;
        uint4 u[sizeof(CellGeo<float>) / 16];
    } U;
    const uint4 *src = reinterpret_cast<const uint4 *>(A.geo + c);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(CellGeo<float>) / 16); ++k) U.u[k] = __ldg(src + k);
    const CellGeo<float> &g = U.g;
    float P[4], t[4], tt = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) P[j] = ox * g.gx[j] + oy * g.gy[j] + oz * g.gz[j];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float sf = ox * g.nx[f] + oy * g.ny[f] + oz * g.nz[f];
        t[f] = ((mask >> f) & 1u) ? fabsf(sf) * (1.f / 12.f) : 0.f;
        tt += t[f];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float w = P[j] + (i == j ? 2.f * (tt - t[i]) : tt - t[i] - t[j]);
            r.W[i][j] = pk(w, w);
        }
    uint32_t up = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        r.t[f] = pk(t[f], t[f]);
        r.nbr[f] = g.nbr[f];
        up |= (((mask >> f) & 1u) && g.nbr[f] >= 0) ? (1u << f) : 0u;
    }
    r.mv = pk(g.mv, g.mv);
    r.c = c;
    r.mask = mask;
    r.code = g.code;
    r.mat = g.mat;
    r.upmask = up;
}

// Groups 2p and 2p+1 of one staged cell: assemble, solve (Gaussian elimination
// without pivoting, negated multipliers so every update is one packed FMA),
// store psi (sorted node order, pair-interleaved).  qrow: the cell's staged
// source row; ups: its staged upwind rows, one per interior inflow face in
// face order; row = G/2 pairs x 32 bytes.
__device__ __forceinline__ void pair_solve(const SweepArgs<float> &A, const TabRow &s, const unsigned char *qrow,
                                           uint32_t row, int p, size_t psi_dir, float ox, float oy, float oz)
{
    const int P = A.G >> 1;
    const f2 sig = *reinterpret_cast<const f2 *>(A.sigma_t + (size_t)s.mat * A.G + 2 * p);
    const f2 mv = s.mv;
    const f2 sv = sig * mv;
    const ulonglong2 *qp = reinterpret_cast<const ulonglong2 *>(qrow + (size_t)p * 32);
    const ulonglong2 q01 = qp[0], q23 = qp[1];
    const f2 qx = {q01.x}, qy = {q01.y}, qz = {q23.x}, qw = {q23.y};
    const f2 qs = (qx + qy) + (qz + qw);
    f2 b[4] = {mv * (qx + qs), mv * (qy + qs), mv * (qz + qs), mv * (qw + qs)};
    const uint32_t c = s.c, code = s.code, upmask = s.upmask, mask = s.mask;
    if (A.S1) {
        const float4 s0 = __ldg(A.S1 + (size_t)c * A.G + 2 * p), s1 = __ldg(A.S1 + (size_t)c * A.G + 2 * p + 1);
        float m0, m1;
        upk(mv, m0, m1);
        const f2 os = pk(5.f * m0 * (ox * s0.x + oy * s0.y + oz * s0.z), 5.f * m1 * (ox * s1.x + oy * s1.y + oz * s1.z));
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = b[i] + os;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!((mask >> f) & 1u)) continue;
        f2 v0, v1, v2;
        if ((upmask >> f) & 1u) {
            const uint32_t slot = __popc(upmask & ((1u << f) - 1u));
            const ulonglong2 *up = reinterpret_cast<const ulonglong2 *>(qrow + (size_t)(1 + slot) * row + (size_t)p * 32);
            const ulonglong2 u01 = up[0], u23 = up[1];
            const f2 ux = {u01.x}, uy = {u01.y}, uz = {u23.x}, uw = {u23.y};
            const uint32_t fn = (code >> (2 * f)) & 3u;
            v0 = sel2(fn == 0u, uy, ux);
            v1 = sel2(fn <= 1u, uz, uy);
            v2 = sel2(fn <= 2u, uw, uz);
        } else if (A.psi_in) {
            const int4 tv = __ldg(A.tets + c);
            const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
            const float *pi = A.psi_in;
            v0 = *reinterpret_cast<const f2 *>(pi + (size_t)vi[f == 0 ? 1 : 0] * A.G + 2 * p);
            v1 = *reinterpret_cast<const f2 *>(pi + (size_t)vi[f <= 1 ? 2 : 1] * A.G + 2 * p);
            v2 = *reinterpret_cast<const f2 *>(pi + (size_t)vi[f <= 2 ? 3 : 2] * A.G + 2 * p);
        } else {
            continue;  // vacuum
        }
        const f2 Uf = (v0 + v1) + v2;
        const f2 tf = s.t[f];
        const int i0 = f == 0 ? 1 : 0, i1 = f <= 1 ? 2 : 1, i2 = f <= 2 ? 3 : 2;
        b[i0] = fma2(tf, v0 + Uf, b[i0]);
        b[i1] = fma2(tf, v1 + Uf, b[i1]);
        b[i2] = fma2(tf, v2 + Uf, b[i2]);
    }
    const f2 two = pk(2.f, 2.f);
    f2 a[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = i == j ? fma2(two, sv, s.W[i][i]) : s.W[i][j] + sv;
    // elimination with n_ik = -a_ik / a_kk
    const f2 nr0 = nrcp2(a[0][0]);
    const f2 n10 = a[1][0] * nr0, n20 = a[2][0] * nr0, n30 = a[3][0] * nr0;
    const f2 a11 = fma2(n10, a[0][1], a[1][1]), a12 = fma2(n10, a[0][2], a[1][2]), a13 = fma2(n10, a[0][3], a[1][3]);
    const f2 a21 = fma2(n20, a[0][1], a[2][1]), a22 = fma2(n20, a[0][2], a[2][2]), a23 = fma2(n20, a[0][3], a[2][3]);
    const f2 a31 = fma2(n30, a[0][1], a[3][1]), a32 = fma2(n30, a[0][2], a[3][2]), a33 = fma2(n30, a[0][3], a[3][3]);
    const f2 b1 = fma2(n10, b[0], b[1]), b2 = fma2(n20, b[0], b[2]), b3 = fma2(n30, b[0], b[3]);
    const f2 nr1 = nrcp2(a11);
    const f2 n21 = a21 * nr1, n31 = a31 * nr1;
    const f2 c22 = fma2(n21, a12, a22), c23 = fma2(n21, a13, a23), c32 = fma2(n31, a12, a32), c33 = fma2(n31, a13, a33);
    const f2 d2 = fma2(n21, b1, b2), d3 = fma2(n31, b1, b3);
    const f2 nr2 = nrcp2(c22);
    const f2 n32 = c32 * nr2;
    const f2 e33 = fma2(n32, c23, c33), e3 = fma2(n32, d2, d3);
    // back substitution on y = -x:  y_k = (b_k + sum_{j>k} a_kj y_j) * (-1/a_kk)
    const f2 y3 = e3 * nrcp2(e33);
    const f2 y2 = fma2(c23, y3, d2) * nr2;
    const f2 y1 = fma2(a13, y3, fma2(a12, y2, b1)) * nr1;
    const f2 y0 = fma2(a[0][3], y3, fma2(a[0][2], y2, fma2(a[0][1], y1, b[0]))) * nr0;
    const f2 m1 = pk(-1.f, -1.f);
    P4 o;
    o.x = y0 * m1;
    o.y = y1 * m1;
    o.z = y2 * m1;
    o.w = y3 * m1;
    st_pair(reinterpret_cast<float *>(A.psi) + ((psi_dir + (size_t)c) * P + p) * 8, o);
}

// Shared memory of one warp on the paired path: the cell table and three stage
// buffers (each: cps cells x [source row, 3 upwind rows]); the mbarriers come on top.
struct PairLayout {
    uint32_t P, row, cps, lpc_shift, ppl, stage, table, ns;
    __device__ __host__ PairLayout(int G, int max_cells, int stages = 3) : ns((uint32_t)stages)
    {
        P = (uint32_t)G / 2;
        row = P * 32u;
        lpc_shift = 0;  // lanes per cell: the smallest power of two >= min(P, 32)
        while ((1u << lpc_shift) < (P >= 32u ? 32u : P)) ++lpc_shift;
        cps = 32u >> lpc_shift;        // cells per stage
        ppl = (P + 31u) / 32u;         // pair slots per lane
        stage = cps * 4u * row;
        table = (uint32_t)max_cells * (uint32_t)sizeof(TabRow);
    }
    __device__ __host__ uint32_t bytes() const { return table + ns * stage; }
};

// One task on the paired path.  Lanes first build the task's cell table in
// parallel (lane j: cell j), then the stages (cps cells each) stream through
// a ring of A.stages (2 or 3) buffers of bulk asynchronous copies while lanes solve pairs:
// lane l takes cell l >> lpc_shift of the stage and pairs (l mod lpc) + 32 m.
// Returns false if a wait ran out (error word set).
__device__ __forceinline__ bool run_task_pairs(const SweepArgs<float> &A, uint4 ti, int lane, float ox, float oy,
                                               float oz, size_t psi_dir, unsigned char *wsm, uint64_t *bars,
                                               uint32_t &ph, unsigned long long *wacc)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t ncell = ti.y & 0xffffu;
    const PairLayout L(A.G, A.max_cells, A.stages);
    TabRow *tab = reinterpret_cast<TabRow *>(wsm);
    unsigned char *stages = wsm + L.table;
    for (uint32_t j = lane; j < ncell; j += 32) tab_setup(A, __ldg(A.cells + ti.x + j), ox, oy, oz, tab[j]);
    __syncwarp();
    const uint32_t nst = (ncell + L.cps - 1) / L.cps;
    // psi rows written by other warps (generic proxy, acquired through the queue)
    // are read below by the async proxy
    fence_proxy_async_global();
    auto issue = [&](uint32_t st) {
        const uint32_t b = st % L.ns, k0 = st * L.cps;
        const uint32_t k = k0 + (uint32_t)lane;
        const bool mine = (uint32_t)lane < L.cps && k < ncell;
        uint32_t upm = mine ? tab[k].upmask : 0u;
        if (__popc(upm) > 3) {  // a closed tetrahedron has at most three inflow faces
            atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
            upm = 0u;
        }
        const uint32_t rows = mine ? 1u + __popc(upm) : 0u;
        const uint32_t bytes = __reduce_add_sync(FULL, rows) * L.row;
        if (lane == 0) {
            fence_proxy_async_shared();  // earlier generic reads of this buffer come first
            mbar_arrive_expect_tx(&bars[b], bytes);
        }
        __syncwarp();
        if (mine) {
            unsigned char *dst = stages + b * L.stage + (size_t)lane * 4u * L.row;
            const TabRow &r = tab[k];
            bulk_g2s(dst, reinterpret_cast<const float *>(A.q) + (size_t)r.c * L.P * 8, L.row, &bars[b]);
            uint32_t slot = 1;
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if ((upm >> f) & 1u) {
                    bulk_g2s(dst + slot * L.row, reinterpret_cast<const float *>(A.psi) + (psi_dir + (size_t)r.nbr[f]) * L.P * 8,
                             L.row, &bars[b]);
                    ++slot;
                }
        }
    };
    issue(0);
    if (L.ns == 3u && nst > 1) issue(1);
    for (uint32_t st = 0; st < nst; ++st) {
        if (st + L.ns - 1u < nst) issue(st + L.ns - 1u);
        const uint32_t b = st % L.ns;
        if (!mbar_wait(&bars[b], (ph >> b) & 1u, A.wait_limit_ns, &A.ctrl->error, wacc)) return false;
        ph ^= 1u << b;
        const uint32_t j = (uint32_t)lane >> L.lpc_shift, k = st * L.cps + j;
        if (k < ncell) {
            const unsigned char *qrow = stages + b * L.stage + (size_t)j * 4u * L.row;
            const uint32_t p0 = (uint32_t)lane & ((1u << L.lpc_shift) - 1u);
            for (uint32_t m = 0; m < L.ppl; ++m) {
                const uint32_t pp = p0 + 32u * m;
                if (pp < L.P) pair_solve(A, tab[k], qrow, L.row, (int)pp, psi_dir, ox, oy, oz);
            }
        }
        __syncwarp();
    }
    return true;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Staged path with the groups-per-lane count unrolled for the common G = 32 and 64.
template <class T, int NS = 3>
__device__ __forceinline__ bool run_task_staged_any(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                                    size_t psi_dir, unsigned char *wsm, uint64_t *bars, uint32_t &ph,
                                                    unsigned long long *wacc)
{
    if (A.G == 64) return run_task_staged<T, 2, NS>(A, ti, lane, ox, oy, oz, psi_dir, wsm, bars, ph, wacc);
    if (A.G == 32) return run_task_staged<T, 1, NS>(A, ti, lane, ox, oy, oz, psi_dir, wsm, bars, ph, wacc);
    return run_task_staged<T, 0, NS>(A, ti, lane, ox, oy, oz, psi_dir, wsm, bars, ph, wacc);
}

#include "p2_solve.cuh"
#include "p3_solve.cuh"
#include "hex_solve.cuh"

// Persistent sweep: a warp claims a ticket (the next queue slot), waits until
// that slot holds a ready task, executes it with lanes spanning (cell, group)
// units, then decrements the counters of the task's downwind blocks; a
// decrement that reaches zero makes that block ready (work-first generation,
// Algorithm 1; atomic counters, Sec. 3.5).  The warp keeps up to keep_max of
// the blocks it made ready and runs them next, without the queue; it enqueues
// the others.
// Termination: a warp whose ticket is >= n_tasks, or that waits while all
// n_tasks tasks are complete, exits.  Every wait is bounded by wait_limit_ns.
// MODE: 0 = any group count (registers), 1 = G a multiple of 32 (registers),
// 2 = G a multiple of 32 with the rows staged in shared memory (three stages),
// 3 = FP32 and G even: packed group pairs (pair-interleaved source and psi rows),
// 4 = as 2 with two stages and six resident CTAs per SM (FP32),
// 5 = the second-order (ten-node) element, lanes over (cell, group) units,
// 6 = the second-order element staged in shared memory (FP32, G a multiple of 32),
// 7 = the third-order element, four lanes per unit with the system in registers and the
//     cell's group-independent matrix and the element tables in shared memory,
// 8 = trilinear hexahedra, lanes over (cell, group) units,
// 9 = trilinear hexahedra with the group-independent matrices formed once per cell in shared memory (G >= 8).
template <class T, int MODE>
__global__ void __launch_bounds__(128, MODE == 7 ? (sizeof(T) == 4 ? 3 : 2) : MODE == 5 ? 2 : MODE == 6 ? 3 : MODE == 4 ? 6 : MODE == 9 ? (sizeof(T) == 4 ? 4 : 2) : MODE == 8 ? (sizeof(T) == 4 ? 3 : 2) : (sizeof(T) == 4 ? 4 : 3))
    sweep_kernel(const SweepArgs<T> A)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const unsigned epoch = *(const volatile unsigned *)&A.ctrl->epoch;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *wsm = dsm + (size_t)(threadIdx.x >> 5) * A.warp_smem;
    uint32_t ph = 0;  // mbarrier phase parities of this warp's stages
    // the six mbarriers of the staged paths sit in the last 48 bytes of the warp's region
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + A.warp_smem - 48);
    if constexpr (MODE == 2 || MODE == 3 || MODE == 4 || MODE == 6) {
        if (lane == 0) {
            for (int b = 0; b < 6; ++b) mbar_init(&bars[b], 1);
            fence_proxy_async_shared();
        }
        __syncwarp();
    }
    // third order: the element tables sit in shared memory after the warps' regions
    const P3Dev<T> *p3s = reinterpret_cast<const P3Dev<T> *>(dsm + (size_t)(blockDim.x >> 5) * A.warp_smem);
    if constexpr (MODE == 7) {
        p3_stage_tables<T>(A.p3tab, dsm + (size_t)(blockDim.x >> 5) * A.warp_smem);
        __syncthreads();
    }
    // per-warp counters live in shared memory (lane 0 updates them) to spare registers
    __shared__ unsigned long long wstat[8][7];  // polls, wait_ns, busy_ns, done, depth, pops, data-wait cycles
    unsigned long long *ws = wstat[threadIdx.x >> 5];
    if (lane < 7) ws[lane] = 0;
    __syncwarp();
    const unsigned long long t_start = globaltimer();
    // A warp that releases downwind tasks keeps up to keep_max of them on a small
    // private stack and runs them next, most recent first (their upwind rows were
    // just written and are still in L2); it claims a queue ticket only when the
    // stack is empty.  Fewer than n_tasks slots are then filled, so a waiting warp
    // also stops once every task is complete.
    __shared__ unsigned kstack[4][4];  // [warp][slot]
    unsigned *ks = kstack[threadIdx.x >> 5];
    int nk = 0;  // warp-uniform stack depth
    for (;;) {
        unsigned task = 0;
        if (nk > 0) {
            task = ks[--nk];
        } else {
            int stop = 0;
            if (lane == 0) {
                const unsigned long long ticket = atomicAdd(&A.ctrl->head, 1ull);
                const unsigned long long t0 = globaltimer();
                unsigned long long v = 0;
                if (ticket >= A.n_tasks) {
                    stop = 2;
                } else {
                    v = ld_acquire(A.slots + ticket);
                    if ((unsigned)(v >> 32) != epoch) {
                        unsigned ns = 32;
                        for (;;) {
                            __nanosleep(ns);
                            if (ns < 256) ns <<= 1;
                            ++ws[0];
                            v = ld_acquire(A.slots + ticket);
                            if ((unsigned)(v >> 32) == epoch) break;
                            if (ld_volatile(&A.ctrl->complete) >= A.n_tasks) {
                                stop = 2;
                                break;
                            }
                            if (ld_volatile(&A.ctrl->error)) {
                                stop = 1;
                                break;
                            }
                            if (globaltimer() - t0 > A.wait_limit_ns) {
                                atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_TIMEOUT);
                                stop = 1;
                                break;
                            }
                        }
                    }
                }
                const unsigned long long t1 = globaltimer();
                ws[1] += t1 - t0;
                if (!stop) {
                    const long long dq = (long long)(ld_volatile(&A.ctrl->tail) - ticket);
                    ws[4] += dq > 0 ? (unsigned long long)dq : 0ull;
                    ++ws[5];
                    task = (unsigned)v;
                    if (task < A.task_begin || task >= A.task_end) {
                        atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
                        stop = 1;
                    }
                }
            }
            __syncwarp();
            stop = __shfl_sync(FULL, stop, 0);
            if (stop) break;
            task = __shfl_sync(FULL, task, 0);
        }
        __syncwarp();  // every lane has read its task from the stack before kept tasks are written to it
        unsigned long long tb = 0;
        if (lane == 0) tb = globaltimer();

        const uint4 ti = __ldg(A.task + task);
        const uint32_t dir = ti.y >> 16;
        const V4<T> om = ld_ro(A.omega + dir);
        const size_t psi_dir = (size_t)(dir - (uint32_t)A.dir_begin) * (size_t)A.C;
        if constexpr (MODE == 3) {
            if (!run_task_pairs(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6)) break;
        } else if constexpr (MODE == 2) {
            if (!run_task_staged_any(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6)) break;
        } else if constexpr (MODE == 4) {
            if (!run_task_staged_any<T, 2>(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6)) break;
        } else if constexpr (MODE == 1) {
            run_task_wide(A, ti, lane, om.x, om.y, om.z, psi_dir);
        } else if constexpr (MODE == 5) {
            run_task_p2(A, ti, lane, om.x, om.y, om.z, psi_dir);
        } else if constexpr (MODE == 6) {
            if (!run_task_p2_staged(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6)) break;
        } else if constexpr (MODE == 7) {
            run_task_p3(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, p3s);
        } else if constexpr (MODE == 8) {
            run_task_hex(A, ti, lane, om.x, om.y, om.z, psi_dir);
        } else if constexpr (MODE == 9) {
            run_task_hex_shared(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm);
        } else {
            run_task_generic(A, ti, lane, om.x, om.y, om.z, psi_dir);
        }
        // release: every lane's psi stores are ordered before any counter decrement
        fence_acq_rel_gpu();
        __syncwarp();
        for (uint32_t e0 = 0; e0 < ti.w; e0 += 32) {
            const uint32_t e = e0 + lane;
            uint32_t d = 0;
            bool ready = false;
            if (e < ti.w) {
                d = __ldg(A.down + ti.z + e);
                ready = atom_add_acq_rel(A.counters + d, -1) == 1;
            }
            const unsigned rb = __ballot_sync(FULL, ready);
            // the warp keeps (keep_max - nk) of the tasks it made ready, those with the longest
            // chain of downwind tasks first, so a direction's critical path does not wait in the
            // queue behind the other ready tasks; it queues the others
            const int room = A.keep_max - nk;
            bool kept = false;
            if (A.blevel) {
                uint32_t key = ready ? ((uint32_t)min(__ldg(A.blevel + d), (1 << 25) - 1) << 6) | (uint32_t)(63 - lane)
                                     : 0u;
                const int take = min(room, __popc(rb));
                for (int r = 0; r < take; ++r) {
                    const uint32_t km = __reduce_max_sync(FULL, key);
                    if (key == km) {
                        kept = true;
                        ks[nk + r] = d;
                        key = 0u;
                    }
                }
                nk += take;
            } else {
                // the first (keep_max - nk) ready lanes push their task on the warp's stack
                const int rank = __popc(rb & ((1u << lane) - 1u));
                kept = ready && rank < room;
                if (kept) ks[nk + rank] = d;
                nk += min(room, __popc(rb));
            }
            if (ready && !kept) {
                const unsigned long long slot = atomicAdd(&A.ctrl->tail, 1ull);
                if (slot < A.n_tasks)
                    st_release(A.slots + slot, ((unsigned long long)epoch << 32) | d);
                else  // more releases than tasks: the task graph is inconsistent
                    atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
            }
        }
        __syncwarp();  // kept tasks visible to every lane of the warp
        // admission: the task that brings its group to the threshold releases the next group's seeds
        if (A.window < A.n_groups) {
            int ng = -1;
            if (lane == 0) {
                const int grp = __ldg(A.dir_group + dir);
                const int left = atomicSub(A.group_rem + grp, 1) - 1;
                if (left == __ldg(A.group_admit + grp)) {
                    ng = atomicAdd(&A.ctrl->next_group, 1);
                    if (ng >= A.n_groups) ng = -1;
                }
            }
            ng = __shfl_sync(FULL, ng, 0);
            if (ng >= 0) {
                const uint32_t s0 = __ldg(A.gseed + ng), n = __ldg(A.gseed + ng + 1) - s0;
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&A.ctrl->tail, (unsigned long long)n);
                base = __shfl_sync(FULL, base, 0);
                if (base + n > A.n_tasks) {
                    if (lane == 0) atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
                } else {
                    for (uint32_t i = lane; i < n; i += 32)
                        st_release(A.slots + base + i, ((unsigned long long)epoch << 32) | __ldg(A.seeds + s0 + i));
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(&A.ctrl->complete, 1ull);
            ws[2] += globaltimer() - tb;
            ++ws[3];
        }
    }
    const unsigned long long t_end = globaltimer();
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&A.ctrl->tasks_done, ws[3]);
        atomicAdd(&A.ctrl->polls, ws[0]);
        atomicAdd(&A.ctrl->wait_ns, ws[1]);
        atomicAdd(&A.ctrl->busy_ns, ws[2]);
        atomicAdd(&A.ctrl->depth_sum, ws[4]);
        atomicAdd(&A.ctrl->pops, ws[5]);
        atomicAdd(&A.ctrl->data_wait_cycles, ws[6]);
        atomicMin(&A.ctrl->t_first, t_start);
        atomicMax(&A.ctrl->t_last, t_end);
    }
}

// ------------------------------------------------------------------ batched launch
// The hexahedral tasks of a batch run through calls (not inlined), so that their register
// demand does not raise the batched kernel's for the tetrahedral variants.
template <class T>
__device__ __noinline__ void batch_task_hex(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                            size_t psi_dir, unsigned char *wsm)
{
    if (A.mode == 9)
        run_task_hex_shared(A, ti, lane, ox, oy, oz, psi_dir, wsm);
    else
        run_task_hex(A, ti, lane, ox, oy, oz, psi_dir);
}
// Several independent problems in one persistent launch: their tasks share one
// ticket queue under global ids (problem k owns [offsets[k], offsets[k+1]));
// each task runs with its own problem's arguments and kernel variant, and its
// downwind releases are translated back to global ids.
template <class T> struct BatchArgs {
    const SweepArgs<T> *probs;  // [n] per-problem arguments (queue fields unused)
    const uint32_t *offsets;    // [n + 1]
    int32_t n;
    Ctrl *ctrl;
    unsigned long long *slots;
    unsigned long long n_tasks;
    unsigned long long wait_limit_ns;
    uint32_t warp_smem;
};

// HEX: the batch holds hexahedral problems (their tasks run through batch_task_hex).
template <class T, bool HEX>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 3) sweep_batch_kernel(const BatchArgs<T> B)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const unsigned epoch = *(const volatile unsigned *)&B.ctrl->epoch;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *wsm = dsm + (size_t)(threadIdx.x >> 5) * B.warp_smem;
    uint32_t ph = 0;
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + B.warp_smem - 48);
    if (lane == 0) {
        for (int b = 0; b < 6; ++b) mbar_init(&bars[b], 1);
        fence_proxy_async_shared();
    }
    __shared__ unsigned long long wstat[8][7];
    unsigned long long *ws = wstat[threadIdx.x >> 5];
    if (lane < 7) ws[lane] = 0;
    __syncwarp();
    const unsigned long long t_start = globaltimer();
    unsigned keep = 0xffffffffu;  // a block this warp made ready and runs next (global id)
    for (;;) {
        unsigned gid = keep;
        if (keep == 0xffffffffu) {
            int stop = 0;
            if (lane == 0) {
                const unsigned long long ticket = atomicAdd(&B.ctrl->head, 1ull);
                const unsigned long long t0 = globaltimer();
                unsigned long long v = 0;
                if (ticket >= B.n_tasks) {
                    stop = 2;
                } else {
                    v = ld_acquire(B.slots + ticket);
                    if ((unsigned)(v >> 32) != epoch) {
                        unsigned ns = 32;
                        for (;;) {
                            __nanosleep(ns);
                            if (ns < 256) ns <<= 1;
                            ++ws[0];
                            v = ld_acquire(B.slots + ticket);
                            if ((unsigned)(v >> 32) == epoch) break;
                            if (ld_volatile(&B.ctrl->complete) >= B.n_tasks) {
                                stop = 2;
                                break;
                            }
                            if (ld_volatile(&B.ctrl->error)) {
                                stop = 1;
                                break;
                            }
                            if (globaltimer() - t0 > B.wait_limit_ns) {
                                atomicCAS(&B.ctrl->error, 0, (int)TF_ERR_TIMEOUT);
                                stop = 1;
                                break;
                            }
                        }
                    }
                }
                ws[1] += globaltimer() - t0;
                if (!stop) {
                    ++ws[5];
                    gid = (unsigned)v;
                    if (gid >= B.n_tasks) {
                        atomicCAS(&B.ctrl->error, 0, (int)TF_ERR_DEVICE);
                        stop = 1;
                    }
                }
            }
            __syncwarp();
            stop = __shfl_sync(FULL, stop, 0);
            if (stop) break;
            gid = __shfl_sync(FULL, gid, 0);
        }
        keep = 0xffffffffu;
        unsigned long long tb = 0;
        if (lane == 0) tb = globaltimer();
        // problem owning the global id: offsets ascend, n is small
        int lo = 0, hi = B.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(B.offsets + mid) <= gid) lo = mid; else hi = mid - 1;
        }
        const SweepArgs<T> &A = B.probs[lo];
        const uint32_t base = __ldg(B.offsets + lo);
        const uint32_t task = gid - base + A.task_begin;
        const uint4 ti = __ldg(A.task + task);
        const uint32_t dir = ti.y >> 16;
        const V4<T> om = ld_ro(A.omega + dir);
        const size_t psi_dir = (size_t)(dir - (uint32_t)A.dir_begin) * (size_t)A.C;
        bool ok = true;
        if constexpr (sizeof(T) == 4) {
            if (A.mode == 3) ok = run_task_pairs(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6);
            else if (A.mode == 2) ok = run_task_staged_any(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6);
            else if (A.mode == 4) ok = run_task_staged_any<T, 2>(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6);
            else if (HEX && (A.mode == 9 || A.mode == 8)) batch_task_hex(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm);
            else run_task_generic(A, ti, lane, om.x, om.y, om.z, psi_dir);
        } else {
            if (A.mode == 2) ok = run_task_staged_any(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6);
            else if (A.mode == 4) ok = run_task_staged_any<T, 2>(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, ws + 6);
            else if (HEX && (A.mode == 9 || A.mode == 8)) batch_task_hex(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm);
            else run_task_generic(A, ti, lane, om.x, om.y, om.z, psi_dir);
        }
        if (!ok) break;
        fence_acq_rel_gpu();
        __syncwarp();
        for (uint32_t e0 = 0; e0 < ti.w; e0 += 32) {
            const uint32_t e = e0 + lane;
            uint32_t d = 0;
            bool ready = false;
            if (e < ti.w) {
                d = __ldg(A.down + ti.z + e);
                ready = atom_add_acq_rel(A.counters + d, -1) == 1;
            }
            const unsigned rb = __ballot_sync(FULL, ready);
            // keep the ready task with the longest downwind chain (see sweep_kernel)
            int kl = -1;
            if (e0 == 0 && rb) {
                if (A.blevel) {
                    const uint32_t key = ready ? ((uint32_t)min(__ldg(A.blevel + d), (1 << 25) - 1) << 6) | (uint32_t)(63 - lane)
                                               : 0u;
                    kl = 63 - (int)(__reduce_max_sync(FULL, key) & 63u);
                } else {
                    kl = __ffs(rb) - 1;
                }
            }
            if (kl >= 0) keep = __shfl_sync(FULL, d - A.task_begin + base, kl);
            if (ready && (int)lane != kl) {
                const unsigned long long slot = atomicAdd(&B.ctrl->tail, 1ull);
                if (slot < B.n_tasks)
                    st_release(B.slots + slot, ((unsigned long long)epoch << 32) | (d - A.task_begin + base));
                else
                    atomicCAS(&B.ctrl->error, 0, (int)TF_ERR_DEVICE);
            }
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(&B.ctrl->complete, 1ull);
            ws[2] += globaltimer() - tb;
            ++ws[3];
        }
    }
    const unsigned long long t_end = globaltimer();
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&B.ctrl->tasks_done, ws[3]);
        atomicAdd(&B.ctrl->polls, ws[0]);
        atomicAdd(&B.ctrl->wait_ns, ws[1]);
        atomicAdd(&B.ctrl->busy_ns, ws[2]);
        atomicAdd(&B.ctrl->pops, ws[5]);
        atomicAdd(&B.ctrl->data_wait_cycles, ws[6]);
        atomicMin(&B.ctrl->t_first, t_start);
        atomicMax(&B.ctrl->t_last, t_end);
    }
}
