// Device state and kernels of the S_N sweep (sm_103a).
//
// One transport step (tf_sweep) on the device:
//   source_kernel   q = (Q + sum_g' sigma_s[g'->g] phi_g') / 4 pi          (Eq. (1) right-hand side)
//   for each direction chunk:
//     begin_kernel  new queue epoch, empty queue
//     fill_kernel   dependency counters <- in-degrees; ready slots <- seed tasks
//     sweep_kernel  persistent: warps pull ready (cell block, direction) tasks,
//                   solve the 4x4 upwind-DG systems with lanes over groups,
//                   store psi, and release downwind counters (Algorithm 1, Sec. 3.5)
//     phi_kernel    phi (+)= sum_a w_a psi_a over the chunk                   (Eq. (2))
// Source iteration adds stats_kernel (per-group max and integrated flux,
// Eq. (3)) and residual_kernel (the FP64 stopping test).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tf_internal.h"

namespace tf {

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
    T mv;
    int32_t mat;
    uint32_t code;
    int32_t nbr[4];
};
static_assert(sizeof(CellGeo<float>) == 128, "float cell record must be one 128-byte line");
static_assert(sizeof(CellGeo<double>) % 16 == 0, "double cell record must be 16-byte aligned");

// Queue control block.  head/tail live on their own 128-byte lines.
struct Ctrl {
    unsigned long long head;  // next ticket to claim
    unsigned long long pad0[15];
    unsigned long long tail;  // next slot to fill
    unsigned long long pad1[15];
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
    unsigned long long residual_bits;  // max residual as ordered bits of a non-negative double
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
    const uint32_t *cells;      // (cell << 4) | inflow mask
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

// Bounded wait on an mbarrier phase; false (and the error word set) after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns, int *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > limit_ns) {
            atomicCAS(err, 0, (int)TF_ERR_TIMEOUT);
            return false;
        }
    }
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

// Bytes of shared memory one warp needs for the staged path (3 stages + 6 mbarriers).
template <class T> inline size_t staged_warp_bytes(int G)
{
    return 3 * (sizeof(CellGeo<T>) + 4 * (size_t)G * sizeof(V4<T>)) + 6 * 8;
}

// Lane 0: geometry record and source row of cell c into stage s.
template <class T>
__device__ __forceinline__ void issue_geoq(const SweepArgs<T> &A, unsigned char *st_base, uint64_t *bar, uint32_t c,
                                           const StageLayout<T> &L)
{
    mbar_arrive_expect_tx(bar, (uint32_t)sizeof(CellGeo<T>) + L.row);
    bulk_g2s(st_base, A.geo + c, (uint32_t)sizeof(CellGeo<T>), bar);
    bulk_g2s(st_base + sizeof(CellGeo<T>), A.q + (size_t)c * A.G, L.row, bar);
}

// Lane 0: psi rows of the interior inflow neighbours (mask from the task list,
// neighbours from the staged record) into the stage's upwind slots, in face order.
template <class T>
__device__ __forceinline__ void issue_up(const SweepArgs<T> &A, unsigned char *st_base, uint64_t *bar, uint32_t mask,
                                         size_t psi_dir, const StageLayout<T> &L)
{
    const CellGeo<T> *g = reinterpret_cast<const CellGeo<T> *>(st_base);
    uint32_t n_up = 0;
    int32_t nb[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        nb[f] = g->nbr[f];
        n_up += (((mask >> f) & 1u) && nb[f] >= 0) ? 1u : 0u;
    }
    mbar_arrive_expect_tx(bar, n_up * L.row);
    uint32_t slot = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (((mask >> f) & 1u) && nb[f] >= 0) {
            bulk_g2s(st_base + sizeof(CellGeo<T>) + (1 + slot) * L.row, A.psi + (psi_dir + (size_t)nb[f]) * A.G, L.row,
                     bar);
            ++slot;
        }
    }
}

// Solve every group of one staged cell: lane l takes groups l, l+32, ...
template <class T>
__device__ __forceinline__ void solve_staged_cell(const SweepArgs<T> &A, const unsigned char *st_base, uint32_t entry,
                                                  int lane, T ox, T oy, T oz, size_t psi_dir, const StageLayout<T> &L)
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
    for (int gg = lane; gg < A.G; gg += 32) {
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
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a[i][j] = P[j] + (i == j ? T(2) * (tt - t[i] + sv) : (tt - t[i] - t[j]) + sv);
        T x[4];
        solve4(a, b, x);
        V4<T> o;
        o.x = x[0];
        o.y = x[1];
        o.z = x[2];
        o.w = x[3];
        st_psi(out + gg, o);
    }
}

// One task through the staged pipeline.  Stage of cell k = k mod 3; for each
// stage two mbarriers (geometry+source, upwind rows) whose phase parities are
// kept in `ph` (bit s: geometry barrier of stage s, bit 3+s: upwind barrier).
// Returns false if a wait ran out (error word set).
template <class T>
__device__ __forceinline__ bool run_task_staged(const SweepArgs<T> &A, uint4 ti, int lane, T ox, T oy, T oz,
                                                size_t psi_dir, unsigned char *wsm, uint32_t &ph)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t ncell = ti.y & 0xffffu;
    const StageLayout<T> L(A.G);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + 3 * L.stage);
    const uint32_t e_lo = lane < (int)ncell ? __ldg(A.cells + ti.x + lane) : 0u;
    const uint32_t e_hi = lane + 32 < (int)ncell ? __ldg(A.cells + ti.x + 32 + lane) : 0u;
    auto entry = [&](uint32_t k) { return __shfl_sync(FULL, k < 32 ? e_lo : e_hi, k & 31); };
    // psi rows written by other warps (generic proxy, acquired through the
    // queue) are read here by the async proxy
    if (lane == 0) fence_proxy_async_global();
    const uint32_t e0 = entry(0);
    const uint32_t e1 = ncell > 1 ? entry(1) : 0u;
    if (lane == 0) {
        issue_geoq(A, wsm, &bars[0], e0 >> 4, L);
        if (ncell > 1) issue_geoq(A, wsm + L.stage, &bars[1], e1 >> 4, L);
    }
    if (!mbar_wait(&bars[0], ph & 1u, A.wait_limit_ns, &A.ctrl->error)) return false;
    ph ^= 1u;
    if (lane == 0) issue_up(A, wsm, &bars[3], e0 & 15u, psi_dir, L);
    for (uint32_t k = 0; k < ncell; ++k) {
        const uint32_t s = k % 3u;
        const uint32_t ek = entry(k);
        if (k + 1 < ncell) {
            const uint32_t s1 = (k + 1) % 3u, en = entry(k + 1);
            if (!mbar_wait(&bars[s1], (ph >> s1) & 1u, A.wait_limit_ns, &A.ctrl->error)) return false;
            ph ^= 1u << s1;
            if (lane == 0) issue_up(A, wsm + s1 * L.stage, &bars[3 + s1], en & 15u, psi_dir, L);
        }
        if (k + 2 < ncell) {
            const uint32_t s2 = (k + 2) % 3u, en2 = entry(k + 2);
            if (lane == 0) {
                fence_proxy_async_shared();  // generic reads of this stage (cell k-1) before the async writes
                issue_geoq(A, wsm + s2 * L.stage, &bars[s2], en2 >> 4, L);
            }
        }
        if (!mbar_wait(&bars[3 + s], (ph >> (3 + s)) & 1u, A.wait_limit_ns, &A.ctrl->error)) return false;
        ph ^= 1u << (3 + s);
        solve_staged_cell(A, wsm + s * L.stage, ek, lane, ox, oy, oz, psi_dir, L);
        __syncwarp();
    }
    return true;
}

// ------------------------------------------------------------------ packed pairs
// FP32 mode, even G: a lane solves two groups of one cell at once.  Both
// groups' values of a quantity share one 64-bit register and Blackwell's
// packed FP32 instructions (add/sub/mul/fma .f32x2) operate on both halves.
// The source and psi rows are stored pair-interleaved, [cell][G/2][node][2],
// so one 32-byte load yields the four packed nodal values of a group pair.
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

// Shared memory of one warp on the paired path: the cell table, three stage
// buffers (each: cps cells x [source row, 3 upwind rows]) and their mbarriers.
struct PairLayout {
    uint32_t P, row, cps, lpc_shift, ppl, stage, table;
    __device__ __host__ PairLayout(int G, int max_cells)
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
    __device__ __host__ uint32_t bytes() const { return table + 3u * stage + 3u * 8u; }
};

// One task on the paired path.  Lanes first build the task's cell table in
// parallel (lane j: cell j), then the stages (cps cells each) stream through
// a three-buffer ring of bulk asynchronous copies while lanes solve pairs:
// lane l takes cell l >> lpc_shift of the stage and pairs (l mod lpc) + 32 m.
// Returns false if a wait ran out (error word set).
__device__ __forceinline__ bool run_task_pairs(const SweepArgs<float> &A, uint4 ti, int lane, float ox, float oy,
                                               float oz, size_t psi_dir, unsigned char *wsm, uint32_t &ph)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t ncell = ti.y & 0xffffu;
    const PairLayout L(A.G, A.max_cells);
    TabRow *tab = reinterpret_cast<TabRow *>(wsm);
    unsigned char *stages = wsm + L.table;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stages + 3 * L.stage);
    for (uint32_t j = lane; j < ncell; j += 32) tab_setup(A, __ldg(A.cells + ti.x + j), ox, oy, oz, tab[j]);
    __syncwarp();
    const uint32_t nst = (ncell + L.cps - 1) / L.cps;
    // psi rows written by other warps (generic proxy, acquired through the queue)
    // are read below by the async proxy
    fence_proxy_async_global();
    auto issue = [&](uint32_t st) {
        const uint32_t b = st % 3u, k0 = st * L.cps;
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
    if (nst > 1) issue(1);
    for (uint32_t st = 0; st < nst; ++st) {
        if (st + 2 < nst) issue(st + 2);
        const uint32_t b = st % 3u;
        if (!mbar_wait(&bars[b], (ph >> b) & 1u, A.wait_limit_ns, &A.ctrl->error)) return false;
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

// Persistent sweep: every warp repeatedly claims a ticket (the next queue
// slot), waits until that slot holds a ready task, executes it with lanes
// spanning (cell, group) units, then decrements the counters of the task's
// downwind blocks; the decrement that reaches zero enqueues that block
// (work-first generation, Algorithm 1; atomic counters, Sec. 3.5).
// A warp claims its next ticket as soon as it starts a task, so the claim's
// latency overlaps the task.  Termination: exactly n_tasks slots get filled,
// so a warp whose ticket is >= n_tasks exits.  Every wait is bounded by
// wait_limit_ns.
// MODE: 0 = any group count (registers), 1 = G a multiple of 32 (registers),
// 2 = G a multiple of 32 with the rows staged in shared memory, 3 = FP32 and
// G even: packed group pairs (pair-interleaved source and psi rows).
template <class T, int MODE>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 3) sweep_kernel(const SweepArgs<T> A)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const unsigned epoch = *(const volatile unsigned *)&A.ctrl->epoch;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *wsm = dsm + (size_t)(threadIdx.x >> 5) * A.warp_smem;
    uint32_t ph = 0;  // mbarrier phase parities of this warp's stages
    if constexpr (MODE == 2) {
        if (lane == 0) {
            uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + 3 * StageLayout<T>(A.G).stage);
            for (int b = 0; b < 6; ++b) mbar_init(&bars[b], 1);
            fence_proxy_async_shared();
        }
        __syncwarp();
    }
    if constexpr (MODE == 3) {
        if (lane == 0) {
            const PairLayout L(A.G, A.max_cells);
            uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + L.table + 3 * L.stage);
            for (int b = 0; b < 3; ++b) mbar_init(&bars[b], 1);
            fence_proxy_async_shared();
        }
        __syncwarp();
    }
    // per-warp counters live in shared memory (lane 0 updates them) to spare registers
    __shared__ unsigned long long wstat[8][6];  // polls, wait_ns, busy_ns, done, depth, pops
    unsigned long long *ws = wstat[threadIdx.x >> 5];
    if (lane < 6) ws[lane] = 0;
    __syncwarp();
    const unsigned long long t_start = globaltimer();
    unsigned long long ticket = 0;
    if (lane == 0) ticket = atomicAdd(&A.ctrl->head, 1ull);
    ticket = __shfl_sync(FULL, ticket, 0);
    while (ticket < A.n_tasks) {
        unsigned task = 0;
        int stop = 0;
        if (lane == 0) {
            const unsigned long long t0 = globaltimer();
            unsigned long long v = ld_acquire(A.slots + ticket);
            if ((unsigned)(v >> 32) != epoch) {
                unsigned ns = 64;
                for (;;) {
                    __nanosleep(ns);
                    if (ns < 2048) ns <<= 1;
                    ++ws[0];
                    v = ld_acquire(A.slots + ticket);
                    if ((unsigned)(v >> 32) == epoch) break;
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
            const unsigned long long t1 = globaltimer();
            ws[1] += t1 - t0;
            const long long dq = (long long)(ld_volatile(&A.ctrl->tail) - ticket);
            ws[4] += dq > 0 ? (unsigned long long)dq : 0ull;
            ++ws[5];
            task = (unsigned)v;
            if (!stop && (task < A.task_begin || task >= A.task_end)) {
                atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
                stop = 1;
            }
        }
        __syncwarp();
        stop = __shfl_sync(FULL, stop, 0);
        if (stop) break;
        task = __shfl_sync(FULL, task, 0);
        unsigned long long tb = 0;
        if (lane == 0) tb = globaltimer();
        // claim the next ticket now; its latency overlaps this task
        unsigned long long next = 0;
        if (lane == 0) next = atomicAdd(&A.ctrl->head, 1ull);

        const uint4 ti = __ldg(A.task + task);
        const uint32_t dir = ti.y >> 16;
        const V4<T> om = ld_ro(A.omega + dir);
        const size_t psi_dir = (size_t)(dir - (uint32_t)A.dir_begin) * (size_t)A.C;
        if constexpr (MODE == 3) {
            if (!run_task_pairs(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, ph)) break;
        } else if constexpr (MODE == 2) {
            if (!run_task_staged(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, ph)) break;
        } else if constexpr (MODE == 1) {
            run_task_wide(A, ti, lane, om.x, om.y, om.z, psi_dir);
        } else {
            run_task_generic(A, ti, lane, om.x, om.y, om.z, psi_dir);
        }
        // release: every lane's psi stores are ordered before any counter decrement
        fence_acq_rel_gpu();
        __syncwarp();
        for (uint32_t e = lane; e < ti.w; e += 32) {
            const uint32_t d = __ldg(A.down + ti.z + e);
            if (atom_add_acq_rel(A.counters + d, -1) == 1) {
                const unsigned long long slot = atomicAdd(&A.ctrl->tail, 1ull);
                if (slot < A.n_tasks)
                    st_release(A.slots + slot, ((unsigned long long)epoch << 32) | d);
                else  // more releases than tasks: the task graph is inconsistent
                    atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
            }
        }
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
            ws[2] += globaltimer() - tb;
            ++ws[3];
        }
        ticket = __shfl_sync(FULL, next, 0);
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
        atomicMin(&A.ctrl->t_first, t_start);
        atomicMax(&A.ctrl->t_last, t_end);
    }
}

// New launch: bump the epoch, empty the queue.
__global__ void begin_kernel(Ctrl *ctrl, unsigned long long n_seeds, int reset_stats, int first_group)
{
    ctrl->epoch = ctrl->epoch + 1u;
    ctrl->next_group = first_group;
    ctrl->head = 0;
    ctrl->tail = n_seeds;
    if (reset_stats) {
        ctrl->tasks_done = ctrl->polls = ctrl->wait_ns = ctrl->busy_ns = 0;
        ctrl->depth_sum = ctrl->pops = 0;
        ctrl->kernel_ns = 0;
    }
    ctrl->t_first = ~0ull;
    ctrl->t_last = 0;
}

// Counters of the chunk's tasks <- in-degrees; group counters <- group sizes;
// the first n_seeds slots <- the seeds of the initially admitted groups.
__global__ void fill_kernel(Ctrl *ctrl, int *counters, const int *indeg, uint32_t task_begin, uint32_t n_tasks,
                            unsigned long long *slots, const uint32_t *seeds, uint32_t n_seeds, int inject_stall,
                            int *group_rem, const int *group_total, int n_groups)
{
    const unsigned epoch = ctrl->epoch;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_groups; i += gridDim.x * blockDim.x)
        group_rem[i] = group_total[i];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tasks; i += gridDim.x * blockDim.x)
        counters[task_begin + i] = indeg[task_begin + i];
    if (inject_stall) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_seeds; i += gridDim.x * blockDim.x)
        slots[i] = ((unsigned long long)epoch << 32) | seeds[i];
}

__global__ void end_kernel(Ctrl *ctrl)
{
    if (ctrl->t_last > ctrl->t_first) ctrl->kernel_ns += ctrl->t_last - ctrl->t_first;
}

// ============================================================== source update
// q[c][g][j] = (Q[c][g][j] + sum_g' sigma_s[m][g'][g] phi[c][g'][perm(j)]) / (4 pi)
// phi is in the caller's node order; q (and Q, uploaded pre-permuted) are in
// the cell's sorted node order, perm(j) = caller's index of sorted node j.
// One CTA stages the FP64 scalar flux of a few cells (converted to the sweep
// precision) in shared memory; thread (cell, g) forms the 4 nodal sums.
template <class T>
__global__ void __launch_bounds__(256) source_kernel(const double *__restrict__ phi, const V4<T> *__restrict__ Qext,
                                                     const T *__restrict__ sigma_s, const CellGeo<T> *__restrict__ geo,
                                                     V4<T> *__restrict__ q, int64_t C, int G, int cells_per_cta,
                                                     int paired)
{
    extern __shared__ unsigned char smem_raw[];
    T *ph = reinterpret_cast<T *>(smem_raw);  // [cells_per_cta][G][4]
    const T inv4pi = T(1.0 / (4.0 * 3.14159265358979323846));
    for (int64_t c0 = (int64_t)blockIdx.x * cells_per_cta; c0 < C; c0 += (int64_t)gridDim.x * cells_per_cta) {
        const int nc = (int)((C - c0) < (int64_t)cells_per_cta ? (C - c0) : (int64_t)cells_per_cta);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * G * 4; e += blockDim.x) ph[e] = (T)phi[(size_t)c0 * G * 4 + e];
        __syncthreads();
        for (int u = threadIdx.x; u < nc * G; u += blockDim.x) {
            const int lc = u / G, g = u - lc * G;
            const int64_t c = c0 + lc;
            const int m = __ldg(&geo[c].mat);
            const uint32_t code = __ldg(&geo[c].code);
            const T *S = sigma_s + (size_t)m * G * G + g;
            const T *p = ph + (size_t)lc * G * 4;
            T a[4] = {0, 0, 0, 0};
            for (int h = 0; h < G; ++h) {
                const T s = __ldg(S + (size_t)h * G);
                a[0] += s * p[4 * h + 0];
                a[1] += s * p[4 * h + 1];
                a[2] += s * p[4 * h + 2];
                a[3] += s * p[4 * h + 3];
            }
            if (paired) {
                // [c][G/2][node][2]: node j of group g at ((c G/2 + g/2) 4 + j) 2 + (g & 1)
                const size_t base = ((size_t)c * (G >> 1) + (g >> 1)) * 8 + (g & 1);
                const T *Qf = reinterpret_cast<const T *>(Qext) + base;
                T *qf = reinterpret_cast<T *>(q) + base;
#pragma unroll
                for (int j = 0; j < 4; ++j) qf[2 * j] = (__ldg(Qf + 2 * j) + pick4(a, (code >> (8 + 2 * j)) & 3u)) * inv4pi;
            } else {
                const V4<T> Qv = ld_ro(Qext + (size_t)c * G + g);
                V4<T> o;
                o.x = (Qv.x + pick4(a, (code >> 8) & 3u)) * inv4pi;
                o.y = (Qv.y + pick4(a, (code >> 10) & 3u)) * inv4pi;
                o.z = (Qv.z + pick4(a, (code >> 12) & 3u)) * inv4pi;
                o.w = (Qv.w + pick4(a, (code >> 14) & 3u)) * inv4pi;
                q[(size_t)c * G + g] = o;
            }
        }
    }
}

// ============================================================== phi reduction
// phi[c][g][i] (+)= sum over the chunk's directions of w_a psi_a[c][g][i] (Eq. 2).
// Thread per (cell, group); the directions are summed in registers.
// FP32 psi with TF_PHI_PAIR: each product w_a psi is formed exactly as a
// float pair (TwoProd with the weight split into hi + lo) and added with
// TwoSum into a (hi, lo) float pair; the pair is rounded once to FP64.
struct WeightPair {
    float hi, lo;
    double d;
};

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p, float e)
{
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
}

template <class T, bool PAIR>
__global__ void __launch_bounds__(256) phi_kernel(const V4<T> *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                  int Dc, size_t CG, int G, const CellGeo<T> *__restrict__ geo,
                                                  double *__restrict__ phi, int accumulate)
{
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < CG; idx += (size_t)gridDim.x * blockDim.x) {
        double r[4];  // sorted node order
        if constexpr (PAIR) {
            float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            int a = 0;
            for (; a + 4 <= Dc; a += 4) {
                V4<T> v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = ld_stream(psi + (size_t)(a + k) * CG + idx);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const WeightPair w = wts[a + k];
                    const float x[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float p = w.hi * x[i];
                        const float e = fmaf(w.hi, x[i], -p) + w.lo * x[i];
                        two_sum_acc(hi[i], lo[i], p, e);
                    }
                }
            }
            for (; a < Dc; ++a) {
                const V4<T> v = ld_stream(psi + (size_t)a * CG + idx);
                const WeightPair w = wts[a];
                const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float p = w.hi * x[i];
                    const float e = fmaf(w.hi, x[i], -p) + w.lo * x[i];
                    two_sum_acc(hi[i], lo[i], p, e);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = (double)hi[i] + (double)lo[i];
        } else {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int a = 0;
            for (; a + 4 <= Dc; a += 4) {
                V4<T> v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = ld_stream(psi + (size_t)(a + k) * CG + idx);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double w = wts[a + k].d;
                    acc[0] = fma(w, (double)v[k].x, acc[0]);
                    acc[1] = fma(w, (double)v[k].y, acc[1]);
                    acc[2] = fma(w, (double)v[k].z, acc[2]);
                    acc[3] = fma(w, (double)v[k].w, acc[3]);
                }
            }
            for (; a < Dc; ++a) {
                const V4<T> v = ld_stream(psi + (size_t)a * CG + idx);
                const double w = wts[a].d;
                acc[0] = fma(w, (double)v.x, acc[0]);
                acc[1] = fma(w, (double)v.y, acc[1]);
                acc[2] = fma(w, (double)v.z, acc[2]);
                acc[3] = fma(w, (double)v.w, acc[3]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = acc[i];
        }
        // back to the caller's node order: caller node perm(j) <- sorted node j
        const uint32_t code = __ldg(&geo[idx / (size_t)G].code);
        double o[4];
        scatter4(r, code, o);
        double2 *out = reinterpret_cast<double2 *>(phi + idx * 4);
        if (accumulate) {
            const double2 o0 = out[0], o1 = out[1];
            o[0] += o0.x;
            o[1] += o0.y;
            o[2] += o1.x;
            o[3] += o1.y;
        }
        out[0] = make_double2(o[0], o[1]);
        out[1] = make_double2(o[2], o[3]);
    }
}

// Paired layout (FP32, even G): thread per (cell, group pair); per direction
// one 32-byte load of the pair's 8 nodal values, the same accumulation rules.
template <bool PAIR>
__global__ void __launch_bounds__(256) phi_pair_kernel(const float *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                       int Dc, size_t CP, int G, const CellGeo<float> *__restrict__ geo,
                                                       double *__restrict__ phi, int accumulate)
{
    const int P = G >> 1;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < CP; idx += (size_t)gridDim.x * blockDim.x) {
        double r[8];  // [node j][half h] at 2 j + h, sorted node order
        if constexpr (PAIR) {
            float hi[8], lo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) hi[i] = lo[i] = 0.f;
            for (int a = 0; a < Dc; ++a) {
                const float4 *src = reinterpret_cast<const float4 *>(psi + ((size_t)a * CP + idx) * 8);
                const float4 u = __ldcs(src), v = __ldcs(src + 1);
                const float x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
                const WeightPair w = wts[a];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float pp = w.hi * x[i];
                    const float e = fmaf(w.hi, x[i], -pp) + w.lo * x[i];
                    two_sum_acc(hi[i], lo[i], pp, e);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) r[i] = (double)hi[i] + (double)lo[i];
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) r[i] = 0.0;
            for (int a = 0; a < Dc; ++a) {
                const float4 *src = reinterpret_cast<const float4 *>(psi + ((size_t)a * CP + idx) * 8);
                const float4 u = __ldcs(src), v = __ldcs(src + 1);
                const float x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
                const double w = wts[a].d;
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = fma(w, (double)x[i], r[i]);
            }
        }
        const size_t c = idx / (size_t)P;
        const int p = (int)(idx - c * (size_t)P);
        const uint32_t code = __ldg(&geo[c].code);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double rs[4] = {r[h], r[2 + h], r[4 + h], r[6 + h]};
            double o[4];
            scatter4(rs, code, o);
            double2 *out = reinterpret_cast<double2 *>(phi + ((size_t)c * G + 2 * p + h) * 4);
            if (accumulate) {
                const double2 o0 = out[0], o1 = out[1];
                o[0] += o0.x;
                o[1] += o0.y;
                o[2] += o1.x;
                o[3] += o1.y;
            }
            out[0] = make_double2(o[0], o[1]);
            out[1] = make_double2(o[2], o[3]);
        }
    }
}

// psi of one direction, paired layout -> [C][G][4] in the caller's node order.
__global__ void psi_unpair_kernel(const float *__restrict__ src, float4 *__restrict__ dst, size_t CP, int G,
                                  const CellGeo<float> *__restrict__ geo)
{
    const int P = G >> 1;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < CP; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx / (size_t)P;
        const int p = (int)(idx - c * (size_t)P);
        const uint32_t code = __ldg(&geo[c].code);
        const float *s8 = src + idx * 8;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float r[4] = {s8[h], s8[2 + h], s8[4 + h], s8[6 + h]};
            float o[4];
            scatter4(r, code, o);
            dst[(size_t)c * G + 2 * p + h] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

// psi of one direction from sorted to the caller's node order (inspection only).
template <class T>
__global__ void psi_unsort_kernel(const V4<T> *__restrict__ src, V4<T> *__restrict__ dst, size_t CG, int G,
                                  const CellGeo<T> *__restrict__ geo)
{
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < CG; idx += (size_t)gridDim.x * blockDim.x) {
        const uint32_t code = __ldg(&geo[idx / (size_t)G].code);
        const V4<T> v = src[idx];
        const T r[4] = {v.x, v.y, v.z, v.w};
        T o[4];
        scatter4(r, code, o);
        V4<T> w;
        w.x = o[0];
        w.y = o[1];
        w.z = o[2];
        w.w = o[3];
        dst[idx] = w;
    }
}

// ============================================================== FP64 statistics
// Deterministic per-group reductions over cells.  CTA = 32 x 8 threads:
// threadIdx.x walks groups, threadIdx.y walks cells; per-CTA partials go to
// scratch [nblk][G][3] = (max |phi|, sum_c (V_c/4) sum_i phi, sum_c sum_i phi),
// then finish_stats_kernel reduces over CTAs in a fixed order (Eq. (3)) into
// [G][4] = (max, integrated flux, plain nodal sum, 1/max).
__global__ void __launch_bounds__(256) stats_kernel(const double *__restrict__ phi, const double *__restrict__ vol4,
                                                    int64_t C, int G, double *__restrict__ part)
{
    __shared__ double sh[3][8][32];
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + threadIdx.x;
        double mx = 0.0, iv = 0.0, pl = 0.0;
        if (g < G) {
            for (int64_t c = (int64_t)blockIdx.x * 8 + threadIdx.y; c < C; c += (int64_t)gridDim.x * 8) {
                const double2 *p = reinterpret_cast<const double2 *>(phi + ((size_t)c * G + g) * 4);
                const double2 a = p[0], b = p[1];
                const double s = (a.x + a.y) + (b.x + b.y);
                mx = fmax(mx, fmax(fmax(fabs(a.x), fabs(a.y)), fmax(fabs(b.x), fabs(b.y))));
                iv += vol4[c] * s;
                pl += s;
            }
        }
        sh[0][threadIdx.y][threadIdx.x] = mx;
        sh[1][threadIdx.y][threadIdx.x] = iv;
        sh[2][threadIdx.y][threadIdx.x] = pl;
        __syncthreads();
        if (threadIdx.y == 0 && g < G) {
            double m = sh[0][0][threadIdx.x], a = sh[1][0][threadIdx.x], b = sh[2][0][threadIdx.x];
            for (int y = 1; y < 8; ++y) {
                m = fmax(m, sh[0][y][threadIdx.x]);
                a += sh[1][y][threadIdx.x];
                b += sh[2][y][threadIdx.x];
            }
            double *o = part + ((size_t)blockIdx.x * G + g) * 3;
            o[0] = m;
            o[1] = a;
            o[2] = b;
        }
        __syncthreads();
    }
}

__global__ void finish_stats_kernel(const double *__restrict__ part, int nblk, int G, double *__restrict__ out)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double m = 0.0, a = 0.0, b = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double *p = part + ((size_t)k * G + g) * 3;
            m = fmax(m, p[0]);
            a += p[1];
            b += p[2];
        }
        out[4 * g + 0] = m;
        out[4 * g + 1] = a;
        out[4 * g + 2] = b;
        out[4 * g + 3] = m > 0.0 ? 1.0 / m : 0.0;
    }
}

// Stopping test: max over (c, g, i) of |phi_new - phi_old| / max(|phi_new|, floor gmax_g).
// Difference and denominator are FP64; their quotient, both scaled by the
// group's 1/gmax, is formed in FP32, which only blurs r itself by ~1e-7.
// Same 32 (groups) x 8 (cells) CTA shape as stats_kernel.
__global__ void __launch_bounds__(256) residual_kernel(const double *__restrict__ phi_new, const double *__restrict__ phi_old,
                                                       const double *__restrict__ gstats, int64_t C, int G,
                                                       double floor_frac, Ctrl *ctrl)
{
    float rmax = 0.f;
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + threadIdx.x;
        if (g >= G) continue;
        const double gmax = gstats[4 * g], inv = gstats[4 * g + 3];
        const double floor_ = floor_frac * gmax;
        for (int64_t c = (int64_t)blockIdx.x * 8 + threadIdx.y; c < C; c += (int64_t)gridDim.x * 8) {
            const double2 *pn = reinterpret_cast<const double2 *>(phi_new + ((size_t)c * G + g) * 4);
            const double2 *po = reinterpret_cast<const double2 *>(phi_old + ((size_t)c * G + g) * 4);
            const double2 n0 = pn[0], n1 = pn[1], o0 = po[0], o1 = po[1];
            const double nv[4] = {n0.x, n0.y, n1.x, n1.y}, ov[4] = {o0.x, o0.y, o1.x, o1.y};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const double diff = fabs(nv[i] - ov[i]);
                if (diff == 0.0) continue;
                const double den = fmax(fabs(nv[i]), floor_);
                rmax = fmaxf(rmax, den > 0.0 ? __fdiv_rn((float)(diff * inv), (float)(den * inv)) : INFINITY);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((threadIdx.x & 31) == 0 && rmax > 0.f)
        atomicMax(&ctrl->residual_bits, (unsigned long long)__double_as_longlong((double)rmax));
}

// ============================================================== host side
struct DeviceState {
    int device = 0, sm_count = 0;
    int64_t C = 0, nv = 0;
    int32_t G = 0, D = 0, M = 0;
    bool fp64 = false;
    size_t tsize = 4;  // sizeof(T)
    void *geo = nullptr;
    uint32_t *cells = nullptr;
    uint4 *task = nullptr;
    uint32_t *down = nullptr;
    int *indeg = nullptr;
    int *counters = nullptr;
    unsigned long long *slots = nullptr;
    uint32_t *seeds = nullptr;
    void *omega = nullptr;
    void *sigma_t = nullptr;
    void *sigma_s = nullptr;
    void *Q = nullptr;
    void *S1 = nullptr;
    void *psi_in = nullptr;
    int4 *tets = nullptr;
    void *q = nullptr;
    void *psi = nullptr;
    double *vol4 = nullptr;
    WeightPair *wts = nullptr;
    double *phi_buf[2] = {nullptr, nullptr};
    double *part = nullptr;
    double *gstats = nullptr;  // [G][4] = (max |phi|, integrated flux, nodal sum, 1/max)
    Ctrl *ctrl = nullptr;
    Ctrl *ctrl_host = nullptr;  // pinned
    double *gstats_host = nullptr;  // pinned [G][3]
    int Dc = 0, n_chunks = 0;
    std::vector<int64_t> chunk_task_begin;  // [n_chunks + 1]
    std::vector<int64_t> chunk_seed_begin;  // [n_chunks + 1]
    std::vector<int32_t> chunk_group_begin;  // [n_chunks + 1] into the group arrays
    std::vector<uint32_t> gseed_host;        // [n_groups_total + n_chunks] seed offsets
    int32_t *dir_group = nullptr;
    int32_t *group_rem = nullptr, *group_total = nullptr, *group_admit = nullptr;
    uint32_t *gseed = nullptr;
    int window = 0;
    int64_t max_chunk_tasks = 0;
    int grid = 0, wpc = 0;
    bool staged = false;
    bool paired = false;  // FP32, even G: packed group pairs, pair-interleaved q and psi
    int lpc_shift = 0, ppl = 0;
    int mode = 0;  // sweep kernel variant (see sweep_kernel)
    uint32_t warp_smem = 0;
    int stats_blocks = 0;
    int last_chunk = -1;
    std::vector<void *> allocs;
    // event pairs: [0] source, then per chunk (sweep, phi)
    std::vector<cudaEvent_t> ev_start, ev_stop;
};

namespace {

tf_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? TF_ERR_NOMEM : TF_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define TF_CUDA(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <class P> tf_status dmalloc(DeviceState &d, P **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    d.allocs.push_back(q);
    *p = static_cast<P *>(q);
    return TF_OK;
}

template <class P> tf_status upload(DeviceState &d, P **p, const void *src, size_t bytes)
{
    tf_status s = dmalloc(d, p, bytes);
    if (s != TF_OK) return s;
    if (bytes) TF_CUDA(cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice));
    return TF_OK;
}

// Sorted node order of cell c: s2u[j] = caller's local index of the j-th smallest global vertex.
inline void sorted_order(const int32_t *t, int s2u[4])
{
    for (int j = 0; j < 4; ++j) s2u[j] = j;
    for (int a = 1; a < 4; ++a)
        for (int b = a; b > 0 && t[s2u[b - 1]] > t[s2u[b]]; --b) std::swap(s2u[b - 1], s2u[b]);
}

template <class T> void pack_geometry(const Mesh &m, const int32_t *cell_material, std::vector<CellGeo<T>> &out)
{
    out.resize(m.nc);
    for (int64_t c = 0; c < m.nc; ++c) {
        CellGeo<T> &g = out[c];
        std::memset(&g, 0, sizeof(g));
        const double V = m.vol[c];
        int s2u[4];
        sorted_order(&m.tets[4 * c], s2u);
        uint32_t code = 0;
        for (int j = 0; j < 4; ++j) {
            const int u = s2u[j];
            g.gx[j] = (T)(0.25 * V * m.grad[12 * c + 3 * u + 0]);
            g.gy[j] = (T)(0.25 * V * m.grad[12 * c + 3 * u + 1]);
            g.gz[j] = (T)(0.25 * V * m.grad[12 * c + 3 * u + 2]);
            g.nx[j] = (T)m.normal[12 * c + 3 * u + 0];
            g.ny[j] = (T)m.normal[12 * c + 3 * u + 1];
            g.nz[j] = (T)m.normal[12 * c + 3 * u + 2];
            const int32_t n = m.nbr[4 * c + u];
            g.nbr[j] = n;
            if (n >= 0) {
                int s2u_n[4];
                sorted_order(&m.tets[4 * (int64_t)n], s2u_n);
                const int fu = m.nbr_face[4 * c + u];  // neighbour's caller-order face index
                int fs = 0;
                while (s2u_n[fs] != fu) ++fs;
                code |= (uint32_t)fs << (2 * j);
            }
            code |= (uint32_t)u << (8 + 2 * j);
        }
        g.mv = (T)(V / 20.0);
        g.mat = cell_material[c];
        g.code = code;
    }
}

template <class T> tf_status upload_typed(DeviceState &d, void **p, const double *src, size_t n)
{
    std::vector<T> tmp(n);
    for (size_t i = 0; i < n; ++i) tmp[i] = (T)src[i];
    T *q = nullptr;
    tf_status s = upload(d, &q, tmp.data(), n * sizeof(T));
    *p = q;
    return s;
}

// [n][3] -> [n] x V4 (fourth component zero / weight)
template <class T> tf_status upload_vec3(DeviceState &d, void **p, const double *src, size_t n, const double *w4)
{
    std::vector<V4<T>> tmp(n);
    for (size_t i = 0; i < n; ++i) {
        tmp[i].x = (T)src[3 * i];
        tmp[i].y = (T)src[3 * i + 1];
        tmp[i].z = (T)src[3 * i + 2];
        tmp[i].w = w4 ? (T)w4[i] : T(0);
    }
    V4<T> *q = nullptr;
    tf_status s = upload(d, &q, tmp.data(), n * sizeof(V4<T>));
    *p = q;
    return s;
}

template <class T> tf_status create_typed(Problem &p, DeviceState &d, const int32_t *cell_material, const double *sigma_t,
                                          const double *sigma_s, const double *Q, const double *S1, const double *psi_in)
{
    const Mesh &m = *p.mesh;
    const TaskGraph &g = p.graph;
    tf_status s;
    {
        std::vector<CellGeo<T>> geo;
        pack_geometry<T>(m, cell_material, geo);
        CellGeo<T> *gp = nullptr;
        if ((s = upload(d, &gp, geo.data(), geo.size() * sizeof(CellGeo<T>))) != TF_OK) return s;
        d.geo = gp;
    }
    if ((s = upload_vec3<T>(d, &d.omega, p.quad->omega.data(), d.D, p.quad->w.data())) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_t, sigma_t, (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_s, sigma_s, (size_t)d.M * d.G * d.G)) != TF_OK) return s;
    {
        std::vector<double> Qs((size_t)d.C * d.G * 4);
        for (int64_t c = 0; c < d.C; ++c) {
            int s2u[4];
            sorted_order(&m.tets[4 * c], s2u);
            for (int gq = 0; gq < d.G; ++gq)
                for (int j = 0; j < 4; ++j) {
                    const size_t at = d.paired ? (((size_t)c * (d.G / 2) + gq / 2) * 4 + j) * 2 + (gq & 1)
                                               : ((size_t)c * d.G + gq) * 4 + j;
                    Qs[at] = Q[((size_t)c * d.G + gq) * 4 + s2u[j]];
                }
        }
        if ((s = upload_typed<T>(d, &d.Q, Qs.data(), Qs.size())) != TF_OK) return s;
    }
    if (S1) {
        if ((s = upload_vec3<T>(d, &d.S1, S1, (size_t)d.C * d.G, nullptr)) != TF_OK) return s;
    }
    if (psi_in) {
        if ((s = upload_typed<T>(d, &d.psi_in, psi_in, (size_t)d.nv * d.G)) != TF_OK) return s;
        std::vector<int32_t> ts(4 * (size_t)m.nc);
        for (int64_t c = 0; c < m.nc; ++c) {
            int s2u[4];
            sorted_order(&m.tets[4 * c], s2u);
            for (int j = 0; j < 4; ++j) ts[4 * c + j] = m.tets[4 * c + s2u[j]];
        }
        if ((s = upload(d, &d.tets, ts.data(), sizeof(int4) * m.nc)) != TF_OK) return s;
    }
    (void)g;
    return TF_OK;
}

}  // namespace

tf_status device_create(Problem &p, const int32_t *cell_material, const double *sigma_t, const double *sigma_s,
                        const double *Q, const double *S1, const double *psi_in)
{
    DeviceState *dp = new (std::nothrow) DeviceState();
    if (!dp) return fail(TF_ERR_NOMEM, "device state allocation failed");
    p.dev = dp;
    DeviceState &d = *dp;
    const Mesh &m = *p.mesh;
    const TaskGraph &g = p.graph;
    d.device = p.opt.device;
    int ndev = 0;
    TF_CUDA(cudaGetDeviceCount(&ndev));
    if (d.device < 0 || d.device >= ndev) return fail(TF_ERR_ARG, "tf_problem_create: no such CUDA device");
    TF_CUDA(cudaSetDevice(d.device));
    TF_CUDA(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, d.device));
    d.C = m.nc;
    d.nv = m.nv;
    d.G = p.G;
    d.D = p.quad->D;
    d.M = p.M;
    d.fp64 = p.opt.precision == TF_FP64;
    // pairing 0 = automatic: packed pairs unless G is a multiple of 32 (there the
    // shared-memory staged path is faster); 2 = packed pairs whenever G is even
    d.paired = !d.fp64 && d.G % 2 == 0 && (p.opt.pairing == 2 || (p.opt.pairing == 0 && d.G % 32 != 0)) &&
               g.cells_per_task <= 32 &&
               PairLayout(d.G, g.cells_per_task).bytes() <= 227u * 1024u;
    d.tsize = d.fp64 ? 8 : 4;
    const int64_t T = g.T();
    if ((uint64_t)g.down_list.size() >= (1ull << 32)) return fail(TF_ERR_ARG, "graph too large: 2^32 downwind edges");
    tf_status s;
    // task graph
    {
        // inflow masks of the task cell lists, caller face order -> sorted face order
        std::vector<uint8_t> remap((size_t)m.nc * 16);
        for (int64_t c = 0; c < m.nc; ++c) {
            int s2u[4];
            sorted_order(&m.tets[4 * c], s2u);
            for (uint32_t mk = 0; mk < 16; ++mk) {
                uint32_t r = 0;
                for (int j = 0; j < 4; ++j) r |= ((mk >> s2u[j]) & 1u) << j;
                remap[16 * c + mk] = (uint8_t)r;
            }
        }
        std::vector<uint32_t> cl(g.cell_list.size());
        for (size_t i = 0; i < cl.size(); ++i) {
            const uint32_t e = g.cell_list[i], c = e >> 4;
            cl[i] = (c << 4) | remap[16 * (size_t)c + (e & 15u)];
        }
        if ((s = upload(d, &d.cells, cl.data(), cl.size() * 4)) != TF_OK) return s;
    }
    {
        std::vector<uint4> ti(T);
        for (int64_t t = 0; t < T; ++t) {
            ti[t].x = g.task_cell_begin[t];
            ti[t].y = (uint32_t)g.task_ncell[t] | ((uint32_t)g.task_dir[t] << 16);
            ti[t].z = (uint32_t)g.down_begin[t];
            ti[t].w = (uint32_t)(g.down_begin[t + 1] - g.down_begin[t]);
        }
        if ((s = upload(d, &d.task, ti.data(), ti.size() * sizeof(uint4))) != TF_OK) return s;
    }
    if ((s = upload(d, &d.down, g.down_list.data(), g.down_list.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.indeg, g.task_indeg.data(), (size_t)T * 4)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.counters, (size_t)T * 4)) != TF_OK) return s;
    // cell volumes / 4 (FP64) for the integrated flux
    {
        std::vector<double> v4(m.nc);
        for (int64_t c = 0; c < m.nc; ++c) v4[c] = 0.25 * m.vol[c];
        if ((s = upload(d, &d.vol4, v4.data(), v4.size() * 8)) != TF_OK) return s;
    }
    s = d.fp64 ? create_typed<double>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in)
               : create_typed<float>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in);
    if (s != TF_OK) return s;
    if ((s = dmalloc(d, &d.q, (size_t)d.C * d.G * 4 * d.tsize)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.phi_buf[0], (size_t)d.C * d.G * 4 * 8)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.phi_buf[1], (size_t)d.C * d.G * 4 * 8)) != TF_OK) return s;
    // per-direction weights
    {
        std::vector<WeightPair> w(d.D);
        for (int a = 0; a < d.D; ++a) {
            w[a].d = p.quad->w[a];
            w[a].hi = (float)w[a].d;
            w[a].lo = (float)(w[a].d - (double)w[a].hi);
        }
        if ((s = upload(d, &d.wts, w.data(), w.size() * sizeof(WeightPair))) != TF_OK) return s;
    }
    // control block and reduction scratch
    if ((s = dmalloc(d, &d.ctrl, sizeof(Ctrl))) != TF_OK) return s;
    TF_CUDA(cudaMemset(d.ctrl, 0, sizeof(Ctrl)));
    TF_CUDA(cudaMallocHost(&d.ctrl_host, sizeof(Ctrl)));
    TF_CUDA(cudaMallocHost(&d.gstats_host, sizeof(double) * 4 * d.G));
    d.stats_blocks = std::max(1, std::min<int>(4 * d.sm_count, (int)((d.C + 7) / 8)));
    if ((s = dmalloc(d, &d.part, sizeof(double) * 3 * d.G * d.stats_blocks)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.gstats, sizeof(double) * 4 * d.G)) != TF_OK) return s;
    // direction chunks: as many directions per launch as the psi budget allows
    const size_t per_dir = (size_t)d.C * d.G * 4 * d.tsize;
    size_t free_b = 0, total_b = 0;
    TF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    double budget = p.opt.psi_budget_gb > 0 ? p.opt.psi_budget_gb * 1e9 : 0.8 * (double)free_b;
    int Dc = p.opt.dir_chunk > 0 ? std::min(p.opt.dir_chunk, d.D) : (int)std::min<double>(d.D, budget / (double)per_dir);
    if (Dc < 1) return fail(TF_ERR_NOMEM, "not enough device memory for one direction of angular flux");
    d.Dc = Dc;
    d.n_chunks = (d.D + Dc - 1) / Dc;
    // Seeds per chunk.  Directions are grouped by octant (sign pattern of Omega,
    // Sec. 2: the angles of an octant share a sweep orientation); a chunk's
    // groups are admitted `window` at a time so that the active wavefronts stay
    // close and their source and face data stay in L2.  Within a group the
    // seeds with the longest remaining critical path come first.
    std::vector<uint32_t> seeds;
    std::vector<int32_t> dir_group(d.D, 0), group_total, group_admit;
    d.chunk_task_begin.assign(d.n_chunks + 1, 0);
    d.chunk_seed_begin.assign(d.n_chunks + 1, 0);
    d.chunk_group_begin.assign(d.n_chunks + 1, 0);
    d.gseed_host.clear();
    auto octant = [&](int a) {
        const double *o = &p.quad->omega[3 * a];
        return (o[0] < 0.0 ? 1 : 0) | (o[1] < 0.0 ? 2 : 0) | (o[2] < 0.0 ? 4 : 0);
    };
    for (int k = 0; k < d.n_chunks; ++k) {
        const int a0 = k * Dc, a1 = std::min(d.D, a0 + Dc);
        const int64_t t0 = g.dir_task_begin[a0], t1 = g.dir_task_begin[a1];
        d.chunk_task_begin[k] = t0;
        d.chunk_task_begin[k + 1] = t1;
        d.max_chunk_tasks = std::max(d.max_chunk_tasks, t1 - t0);
        int present[8] = {0}, local[8];
        for (int a = a0; a < a1; ++a) present[octant(a)] = 1;
        int ngrp = 0;
        for (int o = 0; o < 8; ++o) local[o] = present[o] ? ngrp++ : -1;
        for (int a = a0; a < a1; ++a) dir_group[a] = local[octant(a)];
        d.chunk_group_begin[k] = (int32_t)group_total.size();
        std::vector<int64_t> tot(ngrp, 0);
        for (int a = a0; a < a1; ++a) tot[dir_group[a]] += g.dir_task_begin[a + 1] - g.dir_task_begin[a];
        for (int j = 0; j < ngrp; ++j) {
            group_total.push_back((int32_t)tot[j]);
            group_admit.push_back((int32_t)(tot[j] / 2));
        }
        for (int j = 0; j < ngrp; ++j) {
            d.gseed_host.push_back((uint32_t)seeds.size());
            const size_t sb = seeds.size();
            for (int a = a0; a < a1; ++a) {
                if (dir_group[a] != j) continue;
                for (int64_t t = g.dir_task_begin[a]; t < g.dir_task_begin[a + 1]; ++t)
                    if (g.task_indeg[t] == 0) seeds.push_back((uint32_t)t);
            }
            std::stable_sort(seeds.begin() + sb, seeds.end(),
                             [&](uint32_t x, uint32_t y) { return g.task_blevel[x] > g.task_blevel[y]; });
        }
        d.gseed_host.push_back((uint32_t)seeds.size());
        d.chunk_seed_begin[k + 1] = (int64_t)seeds.size();
    }
    d.chunk_group_begin[d.n_chunks] = (int32_t)group_total.size();
    d.window = p.opt.octant_window > 0 ? p.opt.octant_window : 2;
    if ((s = upload(d, &d.dir_group, dir_group.data(), dir_group.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.group_total, group_total.data(), group_total.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.group_admit, group_admit.data(), group_admit.size() * 4)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.group_rem, group_total.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.gseed, d.gseed_host.data(), d.gseed_host.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.seeds, seeds.data(), seeds.size() * 4)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.slots, (size_t)d.max_chunk_tasks * 8)) != TF_OK) return s;
    TF_CUDA(cudaMemset(d.slots, 0, (size_t)d.max_chunk_tasks * 8));
    if ((s = dmalloc(d, &d.psi, per_dir * Dc)) != TF_OK) return s;
    // persistent grid: resident CTAs per SM x SMs
    d.wpc = p.opt.warps_per_cta > 0 ? std::min(p.opt.warps_per_cta, 4) : 4;  // launch bounds: 128 threads
    {
        const size_t wb = d.fp64 ? staged_warp_bytes<double>(d.G) : staged_warp_bytes<float>(d.G);
        const size_t wb128 = (wb + 127) / 128 * 128;
        d.staged = p.opt.staging == 0 && d.G % 32 == 0 && g.cells_per_task <= 64 && wb128 * d.wpc <= 227 * 1024;
        d.warp_smem = d.staged ? (uint32_t)wb128 : 0u;
    }
    d.mode = d.paired ? 3 : d.staged ? 2 : (d.G % 32 == 0 && g.cells_per_task <= 64 ? 1 : 0);
    if (d.paired) {
        d.staged = false;
        const uint32_t wb = (PairLayout(d.G, g.cells_per_task).bytes() + 127u) / 128u * 128u;
        while (d.wpc > 1 && wb * d.wpc > 227u * 1024u) d.wpc /= 2;
        d.warp_smem = wb;
        const PairLayout L(d.G, g.cells_per_task);
        d.lpc_shift = (int)L.lpc_shift;
        d.ppl = (int)L.ppl;
    }
    const int dyn = (int)(d.warp_smem * d.wpc);
    const void *kfn = d.fp64 ? (d.mode == 2 ? (const void *)sweep_kernel<double, 2>
                                            : d.mode == 1 ? (const void *)sweep_kernel<double, 1> : (const void *)sweep_kernel<double, 0>)
                             : (d.mode == 3   ? (const void *)sweep_kernel<float, 3>
                                : d.mode == 2 ? (const void *)sweep_kernel<float, 2>
                                : d.mode == 1 ? (const void *)sweep_kernel<float, 1>
                                              : (const void *)sweep_kernel<float, 0>);
    if (dyn > 0) TF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    int per_sm = 0;
    TF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * d.wpc, dyn));
    if (p.opt.ctas_per_sm > 0) per_sm = std::min(per_sm, p.opt.ctas_per_sm);
    d.grid = std::max(1, per_sm) * d.sm_count;
    d.ev_start.resize(1 + 2 * d.n_chunks);
    d.ev_stop.resize(1 + 2 * d.n_chunks);
    for (size_t i = 0; i < d.ev_start.size(); ++i) {
        TF_CUDA(cudaEventCreate(&d.ev_start[i]));
        TF_CUDA(cudaEventCreate(&d.ev_stop[i]));
    }
    TF_CUDA(cudaDeviceSynchronize());
    p.stats.launches_per_step = 1 + 5 * (int64_t)d.n_chunks;
    p.stats.n_tasks = T;
    p.stats.n_units = (int64_t)d.C * d.D * d.G;
    p.stats.n_dirs = d.D;
    p.stats.max_level = g.max_level;
    p.stats.n_chunks = d.n_chunks;
    p.stats.grid_ctas = d.grid;
    p.stats.warps_per_cta = d.wpc;
    p.stats.cells_per_task = g.cells_per_task;
    return TF_OK;
}

void device_destroy(Problem &p)
{
    DeviceState *d = p.dev;
    if (!d) return;
    cudaSetDevice(d->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t e : d->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : d->ev_stop) cudaEventDestroy(e);
    for (void *a : d->allocs) cudaFree(a);
    if (d->ctrl_host) cudaFreeHost(d->ctrl_host);
    if (d->gstats_host) cudaFreeHost(d->gstats_host);
    delete d;
    p.dev = nullptr;
}

namespace {

bool is_device_pointer(const void *ptr)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T> tf_status launch_step(Problem &p, const double *phi_in, double *phi_out, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    const size_t CG = (size_t)d.C * d.G;
    // source update
    {
        const int cpc = std::max(1, 256 / d.G);
        const size_t smem = (size_t)cpc * d.G * 4 * sizeof(T);
        const int blocks = (int)std::min<int64_t>((d.C + cpc - 1) / cpc, (int64_t)d.sm_count * 16);
        TF_CUDA(cudaEventRecord(d.ev_start[0], st));
        source_kernel<T><<<blocks, 256, smem, st>>>(phi_in, (const V4<T> *)d.Q, (const T *)d.sigma_s,
                                                    (const CellGeo<T> *)d.geo, (V4<T> *)d.q, d.C, d.G, cpc,
                                                    d.paired ? 1 : 0);
        TF_CUDA(cudaGetLastError());
        TF_CUDA(cudaEventRecord(d.ev_stop[0], st));
    }
    for (int k = 0; k < d.n_chunks; ++k) {
        const int64_t t0 = d.chunk_task_begin[k], t1 = d.chunk_task_begin[k + 1];
        const int a0 = k * d.Dc, a1 = std::min(d.D, a0 + d.Dc);
        const int gb = d.chunk_group_begin[k], ng = d.chunk_group_begin[k + 1] - gb;
        const int win = std::min(d.window, ng);
        // gseed_host of this chunk: ng + 1 offsets starting at index gb + k
        const uint32_t *gs = d.gseed_host.data() + gb + k;
        const uint32_t s0 = gs[0], s_init = gs[win];
        begin_kernel<<<1, 1, 0, st>>>(d.ctrl, (unsigned long long)(s_init - s0), k == 0, win);
        const int fb = (int)std::min<int64_t>(std::max<int64_t>(1, (t1 - t0 + 255) / 256), (int64_t)d.sm_count * 8);
        fill_kernel<<<fb, 256, 0, st>>>(d.ctrl, d.counters, d.indeg, (uint32_t)t0, (uint32_t)(t1 - t0), d.slots,
                                        d.seeds + s0, s_init - s0, p.opt.inject_stall, d.group_rem + gb,
                                        d.group_total + gb, ng);
        SweepArgs<T> A;
        A.geo = (const CellGeo<T> *)d.geo;
        A.cells = d.cells;
        A.task = d.task;
        A.down = d.down;
        A.counters = d.counters;
        A.slots = d.slots;
        A.ctrl = d.ctrl;
        A.q = (const V4<T> *)d.q;
        A.psi = (V4<T> *)d.psi;
        A.sigma_t = (const T *)d.sigma_t;
        A.omega = (const V4<T> *)d.omega;
        A.S1 = (const V4<T> *)d.S1;
        A.psi_in = (const T *)d.psi_in;
        A.tets = d.tets;
        A.C = d.C;
        A.G = d.G;
        A.dir_begin = a0;
        A.task_begin = (uint32_t)t0;
        A.task_end = (uint32_t)t1;
        A.n_tasks = (unsigned long long)(t1 - t0);
        A.wait_limit_ns = (unsigned long long)(p.opt.wait_limit_s * 1e9);
        A.max_cells = p.graph.cells_per_task;
        A.warp_smem = d.warp_smem;
        A.dir_group = d.dir_group;
        A.group_rem = d.group_rem + gb;
        A.group_admit = d.group_admit + gb;
        A.gseed = d.gseed + gb + k;
        A.seeds = d.seeds;
        A.n_groups = ng;
        A.window = win;
        A.lpc_shift = d.lpc_shift;
        A.ppl = d.ppl;
        TF_CUDA(cudaEventRecord(d.ev_start[1 + 2 * k], st));
        const size_t dyn = (size_t)d.warp_smem * d.wpc;
        if constexpr (sizeof(T) == 4) {
            if (d.mode == 3) sweep_kernel<T, 3><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        }
        if (d.mode == 3) {
        } else if (d.mode == 2)
            sweep_kernel<T, 2><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        else if (d.mode == 1)
            sweep_kernel<T, 1><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        else
            sweep_kernel<T, 0><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        TF_CUDA(cudaGetLastError());
        TF_CUDA(cudaEventRecord(d.ev_stop[1 + 2 * k], st));
        end_kernel<<<1, 1, 0, st>>>(d.ctrl);
        const int pb = (int)std::min<size_t>((CG + 255) / 256, (size_t)d.sm_count * 32);
        TF_CUDA(cudaEventRecord(d.ev_start[2 + 2 * k], st));
        if (d.paired) {
            const size_t CP = CG / 2;
            const int pb2 = (int)std::min<size_t>((CP + 255) / 256, (size_t)d.sm_count * 32);
            if (p.opt.phi_accumulate == TF_PHI_PAIR)
                phi_pair_kernel<true><<<pb2, 256, 0, st>>>((const float *)d.psi, d.wts + a0, a1 - a0, CP, d.G,
                                                           (const CellGeo<float> *)d.geo, phi_out, k > 0);
            else
                phi_pair_kernel<false><<<pb2, 256, 0, st>>>((const float *)d.psi, d.wts + a0, a1 - a0, CP, d.G,
                                                            (const CellGeo<float> *)d.geo, phi_out, k > 0);
        } else if (!d.fp64 && p.opt.phi_accumulate == TF_PHI_PAIR)
            phi_kernel<T, true><<<pb, 256, 0, st>>>((const V4<T> *)d.psi, d.wts + a0, a1 - a0, CG, d.G,
                                                    (const CellGeo<T> *)d.geo, phi_out, k > 0);
        else
            phi_kernel<T, false><<<pb, 256, 0, st>>>((const V4<T> *)d.psi, d.wts + a0, a1 - a0, CG, d.G,
                                                     (const CellGeo<T> *)d.geo, phi_out, k > 0);
        TF_CUDA(cudaGetLastError());
        TF_CUDA(cudaEventRecord(d.ev_stop[2 + 2 * k], st));
        d.last_chunk = k;
    }
    return TF_OK;
}

tf_status step(Problem &p, const double *phi_in, double *phi_out, cudaStream_t st)
{
    return p.dev->fp64 ? launch_step<double>(p, phi_in, phi_out, st) : launch_step<float>(p, phi_in, phi_out, st);
}

// Reads the control block after the stream drained; turns a device error into a status.
tf_status collect(Problem &p, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    TF_CUDA(cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    TF_CUDA(cudaStreamSynchronize(st));
    const Ctrl &c = *d.ctrl_host;
    tf_stats &s = p.stats;
    s.tasks_executed = (int64_t)c.tasks_done;
    s.wait_polls = (int64_t)c.polls;
    s.wait_seconds = c.wait_ns * 1e-9;
    s.busy_seconds = c.busy_ns * 1e-9;
    s.kernel_seconds = c.kernel_ns * 1e-9;
    s.mean_ready = c.pops ? (double)c.depth_sum / (double)c.pops : 0.0;
    {
        float ms = 0.f;
        double src = 0.0, sw = 0.0, ph = 0.0;
        TF_CUDA(cudaEventElapsedTime(&ms, d.ev_start[0], d.ev_stop[0]));
        src = ms * 1e-3;
        for (int k = 0; k < d.n_chunks; ++k) {
            TF_CUDA(cudaEventElapsedTime(&ms, d.ev_start[1 + 2 * k], d.ev_stop[1 + 2 * k]));
            sw += ms * 1e-3;
            TF_CUDA(cudaEventElapsedTime(&ms, d.ev_start[2 + 2 * k], d.ev_stop[2 + 2 * k]));
            ph += ms * 1e-3;
        }
        s.source_event_seconds = src;
        s.sweep_event_seconds = sw;
        s.phi_event_seconds = ph;
        s.cum_source_event_seconds += src;
        s.cum_sweep_event_seconds += sw;
        s.cum_phi_event_seconds += ph;
        s.cum_steps += 1;
    }
    if (c.error) {
        const int err = c.error;
        int zero = 0;
        TF_CUDA(cudaMemcpyAsync(&d.ctrl->error, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        TF_CUDA(cudaStreamSynchronize(st));
        return fail((tf_status)err, err == TF_ERR_TIMEOUT ? "sweep: a device wait exceeded the wait limit"
                                                          : "sweep: device reported an out-of-range task");
    }
    if (c.tasks_done != (unsigned long long)p.graph.T())
        return fail(TF_ERR_DEVICE, "sweep: executed " + std::to_string(c.tasks_done) + " of " +
                                       std::to_string(p.graph.T()) + " tasks");
    return TF_OK;
}

}  // namespace

tf_status device_sweep(Problem &p, const double *phi_in, double *phi_out, void *stream)
{
    DeviceState &d = *p.dev;
    TF_CUDA(cudaSetDevice(d.device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)d.C * d.G * 4 * 8;
    const double *in = phi_in;
    double *out = phi_out;
    const bool host_in = !is_device_pointer(phi_in), host_out = !is_device_pointer(phi_out);
    if (host_in) {
        TF_CUDA(cudaMemcpyAsync(d.phi_buf[0], phi_in, bytes, cudaMemcpyHostToDevice, st));
        in = d.phi_buf[0];
    }
    if (host_out) out = d.phi_buf[1];
    tf_status s = step(p, in, out, st);
    if (s != TF_OK) return s;
    if (host_out) TF_CUDA(cudaMemcpyAsync(phi_out, out, bytes, cudaMemcpyDeviceToHost, st));
    return collect(p, st);
}

tf_status device_iterate(Problem &p, double tol, int32_t max_iters, double *phi, tf_iter_info *info, void *stream)
{
    DeviceState &d = *p.dev;
    TF_CUDA(cudaSetDevice(d.device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t CG = (size_t)d.C * d.G;
    const size_t bytes = CG * 4 * 8;
    const bool host = !is_device_pointer(phi);
    double *cur = d.phi_buf[0], *nxt = d.phi_buf[1];
    if (host)
        TF_CUDA(cudaMemcpyAsync(cur, phi, bytes, cudaMemcpyHostToDevice, st));
    else
        TF_CUDA(cudaMemcpyAsync(cur, phi, bytes, cudaMemcpyDeviceToDevice, st));
    double r = INFINITY;
    int it = 0;
    bool conv = false;
    for (it = 1; it <= max_iters; ++it) {
        tf_status s = step(p, cur, nxt, st);
        if (s != TF_OK) return s;
        stats_kernel<<<d.stats_blocks, dim3(32, 8), 0, st>>>(nxt, d.vol4, d.C, d.G, d.part);
        finish_stats_kernel<<<(d.G + 127) / 128, 128, 0, st>>>(d.part, d.stats_blocks, d.G, d.gstats);
        TF_CUDA(cudaMemsetAsync(&d.ctrl->residual_bits, 0, 8, st));
        residual_kernel<<<d.stats_blocks, dim3(32, 8), 0, st>>>(nxt, cur, d.gstats, d.C, d.G, p.opt.residual_floor,
                                                                d.ctrl);
        TF_CUDA(cudaGetLastError());
        s = collect(p, st);
        if (s != TF_OK) return s;
        std::memcpy(&r, &d.ctrl_host->residual_bits, sizeof(double));
        if (info && info->residual_history) info->residual_history[it - 1] = r;
        std::swap(cur, nxt);
        if (r < tol) {
            conv = true;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    // integrated flux of the final phi (already in gstats for the last iterate)
    TF_CUDA(cudaMemcpyAsync(d.gstats_host, d.gstats, sizeof(double) * 4 * d.G, cudaMemcpyDeviceToHost, st));
    if (host)
        TF_CUDA(cudaMemcpyAsync(phi, cur, bytes, cudaMemcpyDeviceToHost, st));
    else
        TF_CUDA(cudaMemcpyAsync(phi, cur, bytes, cudaMemcpyDeviceToDevice, st));
    TF_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = it;
        info->converged = conv ? 1 : 0;
        info->residual = r;
        double tot = 0.0;
        for (int g = 0; g < d.G; ++g) {
            tot += d.gstats_host[4 * g + 1];
            if (info->integrated_flux) info->integrated_flux[g] = d.gstats_host[4 * g + 1];
        }
        info->integrated_total = tot;
    }
    return conv ? TF_OK : fail(TF_ERR_NOT_CONVERGED, "source iteration reached max_iters");
}

tf_status device_psi(Problem &p, int32_t dir, void *out, void *stream)
{
    DeviceState &d = *p.dev;
    if (dir < 0 || dir >= d.D) return fail(TF_ERR_ARG, "tf_problem_psi: direction out of range");
    if (d.last_chunk < 0) return fail(TF_ERR_ARG, "tf_problem_psi: no sweep has run");
    const int a0 = d.last_chunk * d.Dc;
    if (dir < a0 || dir >= std::min(d.D, a0 + d.Dc))
        return fail(TF_ERR_ARG, "tf_problem_psi: direction not in the last swept chunk");
    TF_CUDA(cudaSetDevice(d.device));
    const size_t CG = (size_t)d.C * d.G;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::min<size_t>((CG + 255) / 256, (size_t)d.sm_count * 16);
    if (d.paired)
        psi_unpair_kernel<<<blocks, 256, 0, st>>>((const float *)d.psi + (size_t)(dir - a0) * CG * 4, (float4 *)out,
                                                  CG / 2, d.G, (const CellGeo<float> *)d.geo);
    else if (d.fp64)
        psi_unsort_kernel<double><<<blocks, 256, 0, st>>>((const V4<double> *)d.psi + (size_t)(dir - a0) * CG,
                                                          (V4<double> *)out, CG, d.G, (const CellGeo<double> *)d.geo);
    else
        psi_unsort_kernel<float><<<blocks, 256, 0, st>>>((const V4<float> *)d.psi + (size_t)(dir - a0) * CG,
                                                         (V4<float> *)out, CG, d.G, (const CellGeo<float> *)d.geo);
    TF_CUDA(cudaGetLastError());
    TF_CUDA(cudaStreamSynchronize(st));
    return TF_OK;
}

}  // namespace tf
