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
#include <array>
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tf_internal.h"

namespace tf {

#include "sweep_kernel.cuh"
#include "bsp.h"

// New launch: bump the epoch, empty the queue.
__global__ void begin_kernel(Ctrl *ctrl, unsigned long long n_seeds, int reset_stats, int first_group)
{
    ctrl->epoch = ctrl->epoch + 1u;
    ctrl->next_group = first_group;
    ctrl->head = 0;
    ctrl->tail = n_seeds;
    ctrl->complete = 0;
    if (reset_stats) {
        ctrl->tasks_done = ctrl->polls = ctrl->wait_ns = ctrl->busy_ns = 0;
        ctrl->depth_sum = ctrl->pops = 0;
        ctrl->data_wait_cycles = 0;
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

// psi layout [Dc][C][G] of V4 rows in sorted node order; the result is written
// (or added, for direction chunks after the first) in the caller's node order.
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

// Boundary leakage for the particle balance, per (boundary cell, group) over the
// directions of a chunk: for each boundary face f (sorted face f is opposite sorted
// node f), w_a s_f mean_f(psi_a) on an outflow face (s_f = Omega_a . N_f not below
// the sweep graph's inflow threshold -1e-12 |N_f|) and -w_a |s_f| mean_f(psi_in)
// on an inflow face with prescribed inflow (vacuum: nothing).  FP64 sums, added
// to leak[g].  PAIRED: psi in the pair-interleaved layout [C][G/2][4][2].
template <class T, bool PAIRED>
__global__ void __launch_bounds__(256) leak_kernel(const T *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                   const V4<T> *__restrict__ omega, int Dc, int64_t C, int G,
                                                   const uint32_t *__restrict__ bcells, int64_t nb,
                                                   const CellGeo<T> *__restrict__ geo, const int4 *__restrict__ tets,
                                                   const T *__restrict__ psi_in, double *__restrict__ leak)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nb * G; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = u / G;
        const int g = (int)(u - b * G);
        const uint32_t c = bcells[b];
        const CellGeo<T> &cg = geo[c];
        uint32_t faces = 0;
        T nx[4], ny[4], nz[4], thr[4];
        double pin[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            faces |= (cg.nbr[f] < 0 ? 1u : 0u) << f;
            nx[f] = cg.nx[f];
            ny[f] = cg.ny[f];
            nz[f] = cg.nz[f];
            thr[f] = T(-1e-12) * sqrt(nx[f] * nx[f] + ny[f] * ny[f] + nz[f] * nz[f]);
            pin[f] = 0.0;
        }
        if (psi_in) {
            const int4 tv = tets[c];
            const int vi[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                double m = 0.0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j != f) m += (double)psi_in[(size_t)vi[j] * G + g];
                pin[f] = m / 3.0;
            }
        }
        // FP64 sweeps accumulate in FP64.  FP32 sweeps form each direction's
        // face term in FP32 (its inputs are FP32) and add w_a times it exactly as a
        // float pair (TwoProd, weight split hi + lo; TwoSum), as the phi reduction
        // does: GB300's FP64 rate would make the direction loop FP64-bound.
        double acc = 0.0;
        float hi = 0.f, lo = 0.f;
#pragma unroll 4
        for (int a = 0; a < Dc; ++a) {
            T x[4];
            if constexpr (PAIRED) {
                const T *q = psi + (((size_t)a * C + c) * (G >> 1) + (g >> 1)) * 8 + (g & 1);
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = q[2 * j];
            } else {
                const V4<T> v = reinterpret_cast<const V4<T> *>(psi)[((size_t)a * C + c) * G + g];
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            }
            const T sum = (x[0] + x[1]) + (x[2] + x[3]);
            const V4<T> om = omega[a];
            T t = T(0);  // sum over the boundary faces of s_f mean_f (outflow) or -|s_f| mean_f(psi_in)
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!((faces >> f) & 1u)) continue;
                const T sf = om.x * nx[f] + om.y * ny[f] + om.z * nz[f];
                if (sf >= thr[f]) t += sf * ((sum - x[f]) * T(1.0 / 3.0));
                else t -= fabs(sf) * (T)pin[f];
            }
            if constexpr (sizeof(T) == 8) {
                acc += wts[a].d * (double)t;
            } else {
                const WeightPair w = wts[a];
                const float pp = w.hi * t;
                const float e = fmaf(w.hi, t, -pp) + w.lo * t;
                two_sum_acc(hi, lo, pp, e);
            }
        }
        if constexpr (sizeof(T) == 4) acc = (double)hi + (double)lo;
        atomicAdd(leak + g, acc);
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
// scratch [nblk][G][NP], then the finish kernels reduce over CTAs in a fixed
// order.  Partials: max |phi|, integral sum_c (V_c/4) sum_i phi (Eq. (3)), the
// plain nodal sum, the absorption sum_c sigma_t (V_c/4) sum_i phi and the
// source sum_c (V_c/4) 4 pi sum_i q of the source the sweep used; with the
// stopping test fused, also max |phi_new - phi_old|.
//
// Particle balance per group (summing the rows of every local system, Sigma_i b_i = 1,
// and the directions with their weights; interior faces cancel):
//   R_g = leakage_g + absorption_g - source_g = 0 up to rounding,
// leakage from the phi kernels (boundary faces).  The finish kernels record
// max_g |R_g| / max(source_g, absorption_g) in the control block.
struct BalIn {
    const int32_t *mat;  // [C] material
    const double *sig;   // [M][G] sigma_t (FP64)
    const void *q;       // source rows of the sweep
    int qmode;           // 0: float4 [C][G], 1: FP64 [C][G][4], 2: float pairs [C][G/2][4][2]
    const double *leak;  // [G] boundary leakage
};

__device__ __forceinline__ double q_nodal_sum(const BalIn &b, int64_t c, int g, int G)
{
    if (b.qmode == 0) {
        const float4 v = reinterpret_cast<const float4 *>(b.q)[(size_t)c * G + g];
        return ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
    }
    if (b.qmode == 1) {
        const double2 *v = reinterpret_cast<const double2 *>(b.q) + ((size_t)c * G + g) * 2;
        const double2 x = v[0], y = v[1];
        return (x.x + x.y) + (y.x + y.y);
    }
    const float *f = reinterpret_cast<const float *>(b.q) + ((size_t)c * (G >> 1) + (g >> 1)) * 8 + (g & 1);
    return ((double)f[0] + (double)f[2]) + ((double)f[4] + (double)f[6]);
}

constexpr double kFourPi = 4.0 * 3.14159265358979323846;

// r_g = |R_g| / max(source_g, absorption_g) (0 for a group without source or absorption).
__device__ __forceinline__ void record_balance(double leak, double absorb, double source, Ctrl *ctrl)
{
    const double den = fmax(source, absorb);
    const double r = den > 0.0 ? fabs(leak + absorb - source) / den : 0.0;
    if (r > 0.0) atomicMax(&ctrl->balance_bits, (unsigned long long)__double_as_longlong(r));
}

__global__ void __launch_bounds__(256) stats_kernel(const double *__restrict__ phi, const double *__restrict__ vol4,
                                                    int64_t C, int G, double *__restrict__ part, BalIn bi)
{
    __shared__ double sh[5][8][32];
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + threadIdx.x;
        double mx = 0.0, iv = 0.0, pl = 0.0, ab = 0.0, sr = 0.0;
        if (g < G) {
            for (int64_t c = (int64_t)blockIdx.x * 8 + threadIdx.y; c < C; c += (int64_t)gridDim.x * 8) {
                const double2 *p = reinterpret_cast<const double2 *>(phi + ((size_t)c * G + g) * 4);
                const double2 a = p[0], b = p[1];
                const double s = (a.x + a.y) + (b.x + b.y);
                mx = fmax(mx, fmax(fmax(fabs(a.x), fabs(a.y)), fmax(fabs(b.x), fabs(b.y))));
                iv += vol4[c] * s;
                pl += s;
                ab += bi.sig[(size_t)bi.mat[c] * G + g] * vol4[c] * s;
                sr += vol4[c] * kFourPi * q_nodal_sum(bi, c, g, G);
            }
        }
        sh[0][threadIdx.y][threadIdx.x] = mx;
        sh[1][threadIdx.y][threadIdx.x] = iv;
        sh[2][threadIdx.y][threadIdx.x] = pl;
        sh[3][threadIdx.y][threadIdx.x] = ab;
        sh[4][threadIdx.y][threadIdx.x] = sr;
        __syncthreads();
        if (threadIdx.y == 0 && g < G) {
            double m = sh[0][0][threadIdx.x], a = sh[1][0][threadIdx.x], b = sh[2][0][threadIdx.x];
            double e = sh[3][0][threadIdx.x], f = sh[4][0][threadIdx.x];
            for (int y = 1; y < 8; ++y) {
                m = fmax(m, sh[0][y][threadIdx.x]);
                a += sh[1][y][threadIdx.x];
                b += sh[2][y][threadIdx.x];
                e += sh[3][y][threadIdx.x];
                f += sh[4][y][threadIdx.x];
            }
            double *o = part + ((size_t)blockIdx.x * G + g) * 5;
            o[0] = m;
            o[1] = a;
            o[2] = b;
            o[3] = e;
            o[4] = f;
        }
        __syncthreads();
    }
}

__global__ void finish_stats_kernel(const double *__restrict__ part, int nblk, int G, double *__restrict__ out,
                                    const double *__restrict__ leak, Ctrl *ctrl)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double m = 0.0, a = 0.0, b = 0.0, e = 0.0, f = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double *p = part + ((size_t)k * G + g) * 5;
            m = fmax(m, p[0]);
            a += p[1];
            b += p[2];
            e += p[3];
            f += p[4];
        }
        out[4 * g + 0] = m;
        out[4 * g + 1] = a;
        out[4 * g + 2] = b;
        out[4 * g + 3] = m > 0.0 ? 1.0 / m : 0.0;
        record_balance(leak[g], e, f, ctrl);
    }
}

// Max-norm stopping test fused with the statistics (residual_floor = 1): one
// pass over phi_new and phi_old gives per group max |phi_new|, the integral,
// the nodal sum, the balance sums and max |phi_new - phi_old| (all FP64); the
// finish kernel forms r = max_g max|dphi| / max|phi_new| and the [G][4] statistics.
__global__ void __launch_bounds__(256) stats_res_kernel(const double *__restrict__ phi_new,
                                                        const double *__restrict__ phi_old,
                                                        const double *__restrict__ vol4, int64_t C, int G,
                                                        double *__restrict__ part, BalIn bi)
{
    __shared__ double sh[6][8][32];
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + threadIdx.x;
        double mx = 0.0, iv = 0.0, pl = 0.0, dm = 0.0, ab = 0.0, sr = 0.0;
        if (g < G) {
            for (int64_t c = (int64_t)blockIdx.x * 8 + threadIdx.y; c < C; c += (int64_t)gridDim.x * 8) {
                const double2 *p = reinterpret_cast<const double2 *>(phi_new + ((size_t)c * G + g) * 4);
                const double2 *o = reinterpret_cast<const double2 *>(phi_old + ((size_t)c * G + g) * 4);
                const double2 a = p[0], b = p[1], oa = o[0], ob = o[1];
                const double s = (a.x + a.y) + (b.x + b.y);
                mx = fmax(mx, fmax(fmax(fabs(a.x), fabs(a.y)), fmax(fabs(b.x), fabs(b.y))));
                dm = fmax(dm, fmax(fmax(fabs(a.x - oa.x), fabs(a.y - oa.y)), fmax(fabs(b.x - ob.x), fabs(b.y - ob.y))));
                iv += vol4[c] * s;
                pl += s;
                ab += bi.sig[(size_t)bi.mat[c] * G + g] * vol4[c] * s;
                sr += vol4[c] * kFourPi * q_nodal_sum(bi, c, g, G);
            }
        }
        sh[0][threadIdx.y][threadIdx.x] = mx;
        sh[1][threadIdx.y][threadIdx.x] = iv;
        sh[2][threadIdx.y][threadIdx.x] = pl;
        sh[3][threadIdx.y][threadIdx.x] = dm;
        sh[4][threadIdx.y][threadIdx.x] = ab;
        sh[5][threadIdx.y][threadIdx.x] = sr;
        __syncthreads();
        if (threadIdx.y == 0 && g < G) {
            double m = sh[0][0][threadIdx.x], a = sh[1][0][threadIdx.x], b = sh[2][0][threadIdx.x], d = sh[3][0][threadIdx.x];
            double e = sh[4][0][threadIdx.x], f = sh[5][0][threadIdx.x];
            for (int y = 1; y < 8; ++y) {
                m = fmax(m, sh[0][y][threadIdx.x]);
                a += sh[1][y][threadIdx.x];
                b += sh[2][y][threadIdx.x];
                d = fmax(d, sh[3][y][threadIdx.x]);
                e += sh[4][y][threadIdx.x];
                f += sh[5][y][threadIdx.x];
            }
            double *o = part + ((size_t)blockIdx.x * G + g) * 6;
            o[0] = m;
            o[1] = a;
            o[2] = b;
            o[3] = d;
            o[4] = e;
            o[5] = f;
        }
        __syncthreads();
    }
}

__global__ void finish_stats_res_kernel(const double *__restrict__ part, int nblk, int G, double *__restrict__ out,
                                        const double *__restrict__ leak, Ctrl *ctrl)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double m = 0.0, a = 0.0, b = 0.0, d = 0.0, e = 0.0, f = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double *p = part + ((size_t)k * G + g) * 6;
            m = fmax(m, p[0]);
            a += p[1];
            b += p[2];
            d = fmax(d, p[3]);
            e += p[4];
            f += p[5];
        }
        out[4 * g + 0] = m;
        out[4 * g + 1] = a;
        out[4 * g + 2] = b;
        out[4 * g + 3] = m > 0.0 ? 1.0 / m : 0.0;
        const double r = d == 0.0 ? 0.0 : (m > 0.0 ? d / m : INFINITY);
        if (r > 0.0) atomicMax(&ctrl->residual_bits, (unsigned long long)__double_as_longlong(r));
        record_balance(leak[g], e, f, ctrl);
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

#include "ho_kernels.cuh"

// ============================================================== host side
struct DeviceState {
    int device = 0, sm_count = 0;
    int clock_khz = 0;  // SM clock (kHz), to turn device cycle counts into seconds
    int64_t C = 0, nv = 0;
    int32_t G = 0, D = 0, M = 0;
    bool fp64 = false;
    int order = 1;           // element order: 1 linear (4 nodes), 2 quadratic (10 nodes)
    int nb = 4;              // nodes per cell
    bool hex = false;        // trilinear hexahedra (8 nodes, node-major layouts as the higher orders)
    bool nodemajor() const { return order >= 2 || hex; }
    void *geo2 = nullptr;    // higher orders: P2Geo<T> / P3Geo<T> [C]; hexahedra: HexGeo<T> [C]
    double *hex_pw = nullptr;  // hexahedra: int b_i per cell and node [C][8] (statistics)
    double *vol = nullptr;   // higher orders: cell volumes (FP64)
    void *p3tab = nullptr;   // third order: P3Dev<T> element tables
    double *ho_pw = nullptr;   // higher orders: int phi_i / V [nb]
    int32_t *ho_fn = nullptr;  // higher orders: [4][nodes per face] face nodes
    double *ho_fav = nullptr;  // higher orders: int_f phi / A_f on a face's nodes
    bool two_stage = false;  // staged path with two stages (mode 4)
    bool patches = false;    // spatial-patch tasks: a task's cells may depend on each other
    uint8_t *cells_aux = nullptr;  // patches, staged variants: per cell entry, its in-task upwind handoffs
    int pair_stages = 3;     // paired path: buffers in the ring of staged copies
    size_t tsize = 4;  // sizeof(T)
    void *geo = nullptr;
    uint32_t *cells = nullptr;
    uint4 *task = nullptr;
    uint32_t *down = nullptr;
    int *indeg = nullptr;
    int32_t *blevel = nullptr;  // [T] longest chain of downwind tasks below each task
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
    int32_t *hexv = nullptr;   // hexahedra with prescribed inflow: [C][8] global vertices
    // lagged back edges (hexahedra): per cell entry (lag mask << 26) | first slot; per slot its
    // direction and (cell << 3) | face; the previous step's upwind values [slot][4][G] (T)
    uint32_t *lagw = nullptr;
    uint32_t *lag_slots = nullptr;
    void *lagbuf = nullptr;
    std::vector<int64_t> lag_dir_begin;
    int64_t n_lag = 0;
    void *q = nullptr;
    void *psi = nullptr;
    double *vol4 = nullptr;
    double *leak = nullptr;    // [G] boundary leakage of the last transport step (particle balance)
    uint32_t *bcells = nullptr;  // cells with a boundary face
    int64_t n_bcells = 0;
    int32_t *mat = nullptr;    // [C] material of each cell
    double *sig_d = nullptr;   // [M][G] sigma_t, FP64
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
    std::vector<uint32_t> seeds_host;        // seed task ids, grouped as gseed_host says
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
    uint32_t cta_smem = 0;   // shared memory of the whole CTA after the warps' regions (third-order tables)
    // bulk-synchronous schedules: task ids grouped by (octant, t-level) bucket, per chunk
    int schedule = TF_SCHED_AMT;
    uint32_t *bsp_order = nullptr;
    uint32_t *bsp_bucket = nullptr;          // [n_buckets + 1] offsets into bsp_order
    unsigned int *bsp_bar = nullptr;         // grid-barrier arrival counter
    std::vector<uint32_t> bsp_bucket_host;
    std::vector<int32_t> chunk_bucket_begin;  // [n_chunks + 1]
    int bsp_grid = 0;
    int stats_blocks = 0;
    int last_chunk = -1;
    std::vector<void *> allocs;
    // event pairs: [0] source, then per chunk (sweep, phi)
    std::vector<cudaEvent_t> ev_start, ev_stop;
    // source iteration: one captured graph per ping-pong direction of the phi buffers
    cudaStream_t istream = nullptr;
    cudaEvent_t ev_user = nullptr, ev_done = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graphs_tried = false;
};

namespace {

// Records a timing event; inside a stream capture it becomes an external event
// node of the graph, so replays record it too.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, st);
}

// The dynamic shared-memory limit is an attribute of the kernel function, shared
// by every problem and by captured graphs: it is only ever raised.
cudaError_t ensure_dyn_smem(const void *kfn, int bytes)
{
    static std::mutex mu;
    static std::map<const void *, int> cur;
    std::lock_guard<std::mutex> lk(mu);
    int &c = cur[kfn];
    if (bytes <= c) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) c = bytes;
    return e;
}

tf_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? TF_ERR_NOMEM : TF_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define TF_STR2(x) #x
#define TF_STR(x) TF_STR2(x)
#define TF_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, "sweep.cu:" TF_STR(__LINE__) " " #call); \
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
    if ((s = upload(d, &d.mat, cell_material, sizeof(int32_t) * (size_t)d.C)) != TF_OK) return s;
    if ((s = upload(d, &d.sig_d, sigma_t, sizeof(double) * (size_t)d.M * d.G)) != TF_OK) return s;
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

// Second-order element: cell records (grad lambda, normals, volume, material,
// neighbours, and for each face node the neighbour's local node of the same
// global vertex or edge), cross sections, Q reordered node-major [C][10][G].
template <class T> tf_status create_typed_p2(Problem &p, DeviceState &d, const int32_t *cell_material,
                                             const double *sigma_t, const double *sigma_s, const double *Q)
{
    const Mesh &m = *p.mesh;
    tf_status s;
    {
        auto key = [&](int64_t c, int i) -> std::pair<int32_t, int32_t> {
            const int32_t *t = &m.tets[4 * c];
            if (i < 4) return {t[i], -1};
            const int32_t a = t[p2_edge_end(i - 4, 0)], b = t[p2_edge_end(i - 4, 1)];
            return {std::min(a, b), std::max(a, b)};
        };
        std::vector<P2Geo<T>> geo(m.nc);
        for (int64_t c = 0; c < m.nc; ++c) {
            P2Geo<T> &g = geo[c];
            std::memset(&g, 0, sizeof(g));
            for (int k = 0; k < 12; ++k) {
                g.gl[k] = (T)m.grad[12 * c + k];
                g.nrm[k] = (T)m.normal[12 * c + k];
            }
            g.vol = (T)m.vol[c];
            g.mat = cell_material[c];
            for (int f = 0; f < 4; ++f) {
                const int32_t n = m.nbr[4 * c + f];
                g.nbr[f] = n;
                if (n < 0) continue;
                for (int b = 0; b < 6; ++b) {
                    const auto k = key(c, p2_face_node(f, b));
                    int mm = -1;
                    for (int j = 0; j < 10; ++j)
                        if (key(n, j) == k) mm = j;
                    if (mm < 0) return fail(TF_ERR_MESH, "second-order face node without a match in the neighbour");
                    const int bit = 24 * f + 4 * b;
                    g.fmap[bit >> 5] |= (uint32_t)mm << (bit & 31);
                }
            }
        }
        P2Geo<T> *gp = nullptr;
        if ((s = upload(d, &gp, geo.data(), geo.size() * sizeof(P2Geo<T>))) != TF_OK) return s;
        d.geo2 = gp;
    }
    if ((s = upload_vec3<T>(d, &d.omega, p.quad->omega.data(), d.D, p.quad->w.data())) != TF_OK) return s;
    if ((s = upload(d, &d.mat, cell_material, sizeof(int32_t) * (size_t)d.C)) != TF_OK) return s;
    if ((s = upload(d, &d.sig_d, sigma_t, sizeof(double) * (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_t, sigma_t, (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_s, sigma_s, (size_t)d.M * d.G * d.G)) != TF_OK) return s;
    if ((s = upload(d, &d.vol, m.vol.data(), sizeof(double) * (size_t)d.C)) != TF_OK) return s;
    {
        // statistics and leakage tables: p_i, the face nodes, and the face average (the mean of
        // the three edge nodes: int_f phi_vertex = 0, int_f phi_edge = A_f / 3)
        double pw[10], fav[6] = {0.0, 0.0, 0.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
        int32_t fn[24];
        for (int i = 0; i < 10; ++i) pw[i] = p2_p(i);
        for (int f = 0; f < 4; ++f)
            for (int b = 0; b < 6; ++b) fn[6 * f + b] = p2_face_node(f, b);
        if ((s = upload(d, &d.ho_pw, pw, sizeof(pw))) != TF_OK) return s;
        if ((s = upload(d, &d.ho_fn, fn, sizeof(fn))) != TF_OK) return s;
        if ((s = upload(d, &d.ho_fav, fav, sizeof(fav))) != TF_OK) return s;
    }
    {
        std::vector<double> Qs((size_t)d.C * d.G * 10);
        for (int64_t c = 0; c < d.C; ++c)
            for (int gq = 0; gq < d.G; ++gq)
                for (int i = 0; i < 10; ++i)
                    Qs[((size_t)c * 10 + i) * d.G + gq] = Q[((size_t)c * d.G + gq) * 10 + i];
        if ((s = upload_typed<T>(d, &d.Q, Qs.data(), Qs.size())) != TF_OK) return s;
    }
    return TF_OK;
}

// Trilinear hexahedra: cell records (exact element integrals, integrated face normals,
// material, neighbours and, per face, the neighbour's local vertex of each face node),
// cross sections, the per-cell basis integrals int b_i (row sums of M) for the
// statistics, Q reordered node-major [C][8][G].
template <class T> tf_status create_typed_hex(Problem &p, DeviceState &d, const int32_t *cell_material,
                                              const double *sigma_t, const double *sigma_s, const double *Q, const double *S1,
                                              const double *psi_in)
{
    const Mesh &m = *p.mesh;
    tf_status s;
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 4; ++k)
            if (hex_node(f, k) != hex_face_node(f, k)) return fail(TF_ERR_MESH, "hexahedral face-node tables disagree");
    {
        std::vector<HexGeo<T>> geo(m.nc);
        std::vector<double> pw(8 * (size_t)m.nc);
        for (int64_t c = 0; c < m.nc; ++c) {
            HexGeo<T> &g = geo[c];
            std::memset(&g, 0, sizeof(g));
            g.mat = cell_material[c];
            for (int f = 0; f < 6; ++f) {
                g.nbr[f] = m.nbr[6 * c + f];
                if (g.nbr[f] >= 0)
                    for (int k = 0; k < 4; ++k) {
                        const int v = m.nbr_node[24 * c + 4 * f + k];
                        if (v < 0 || v > 7) return fail(TF_ERR_MESH, "hexahedral face node without a match in the neighbour");
                        g.nmap[f] |= (uint32_t)v << (4 * k);
                    }
                for (int r = 0; r < 3; ++r) g.nbar[f][r] = (T)m.normal[18 * c + 3 * f + r];
                for (int dd = 0; dd < 3; ++dd)
                    for (int k = 0; k < 16; ++k) g.F[f][dd][k] = (T)m.hface[288 * c + 48 * f + 16 * dd + k];
            }
            for (int i = 0; i < 64; ++i) g.M[i] = (T)m.hmass[64 * c + i];
            for (int dd = 0; dd < 3; ++dd)
                for (int i = 0; i < 64; ++i) g.Gd[dd][i] = (T)m.hgrad[192 * c + 64 * dd + i];
            for (int i = 0; i < 8; ++i) {
                double r = 0.0;
                for (int j = 0; j < 8; ++j) r += m.hmass[64 * c + 8 * i + j];
                pw[8 * c + i] = r;
            }
        }
        HexGeo<T> *gp = nullptr;
        if ((s = upload(d, &gp, geo.data(), geo.size() * sizeof(HexGeo<T>))) != TF_OK) return s;
        d.geo2 = gp;
        if ((s = upload(d, &d.hex_pw, pw.data(), pw.size() * sizeof(double))) != TF_OK) return s;
    }
    if ((s = upload_vec3<T>(d, &d.omega, p.quad->omega.data(), d.D, p.quad->w.data())) != TF_OK) return s;
    if ((s = upload(d, &d.mat, cell_material, sizeof(int32_t) * (size_t)d.C)) != TF_OK) return s;
    if ((s = upload(d, &d.sig_d, sigma_t, sizeof(double) * (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_t, sigma_t, (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_s, sigma_s, (size_t)d.M * d.G * d.G)) != TF_OK) return s;
    if ((s = upload(d, &d.vol, m.vol.data(), sizeof(double) * (size_t)d.C)) != TF_OK) return s;
    {
        std::vector<double> Qs((size_t)d.C * d.G * 8);
        for (int64_t c = 0; c < d.C; ++c)
            for (int gq = 0; gq < d.G; ++gq)
                for (int i = 0; i < 8; ++i) Qs[((size_t)c * 8 + i) * d.G + gq] = Q[((size_t)c * d.G + gq) * 8 + i];
        if ((s = upload_typed<T>(d, &d.Q, Qs.data(), Qs.size())) != TF_OK) return s;
    }
    if (S1) {  // [C][G] (x, y, z, 0): the linear anisotropic source Omega.S1, constant over each cell
        if ((s = upload_vec3<T>(d, &d.S1, S1, (size_t)d.C * d.G, nullptr)) != TF_OK) return s;
    }
    if (psi_in) {  // isotropic inflow per boundary vertex and group, and the cells' vertices
        if ((s = upload_typed<T>(d, &d.psi_in, psi_in, (size_t)d.nv * d.G)) != TF_OK) return s;
        if ((s = upload(d, &d.hexv, m.hexes.data(), sizeof(int32_t) * 8 * (size_t)m.nc)) != TF_OK) return s;
    }
    return TF_OK;
}

// Third-order element: cell records (grad lambda, normals, volume, material, neighbours,
// and for each of a face's ten nodes the neighbour's local node at the same place, matched
// by the global vertices its lattice index weights), the exact element tables, cross
// sections, Q reordered node-major [C][20][G].
template <class T> tf_status create_typed_p3(Problem &p, DeviceState &d, const int32_t *cell_material,
                                             const double *sigma_t, const double *sigma_s, const double *Q)
{
    const Mesh &m = *p.mesh;
    tf_status s;
    P3Tables tab;
    p3_element_tables(tab);
    {
        // identity of node i of cell c: its four (global vertex, lattice weight) pairs, sorted
        auto key = [&](int64_t c, int i) {
            int al[4];
            p3_node_alpha(i, al);
            std::array<std::pair<int32_t, int>, 4> k;
            for (int v = 0; v < 4; ++v) k[v] = {al[v] ? m.tets[4 * c + v] : -1, al[v]};
            std::sort(k.begin(), k.end());
            return k;
        };
        std::vector<P3Geo<T>> geo(m.nc);
        for (int64_t c = 0; c < m.nc; ++c) {
            P3Geo<T> &g = geo[c];
            std::memset(&g, 0, sizeof(g));
            for (int k = 0; k < 12; ++k) {
                g.gl[k] = (T)m.grad[12 * c + k];
                g.nrm[k] = (T)m.normal[12 * c + k];
            }
            g.vol = (T)m.vol[c];
            g.mat = cell_material[c];
            for (int f = 0; f < 4; ++f) {
                const int32_t n = m.nbr[4 * c + f];
                g.nbr[f] = n;
                if (n < 0) continue;
                for (int r = 0; r < 10; ++r) {
                    const auto k = key(c, tab.fn[f][r]);
                    int mm = -1;
                    for (int j = 0; j < 20; ++j)
                        if (key(n, j) == k) mm = j;
                    if (mm < 0) return fail(TF_ERR_MESH, "third-order face node without a match in the neighbour");
                    g.fmap[f] |= (unsigned long long)mm << (5 * r);
                }
            }
        }
        P3Geo<T> *gp = nullptr;
        if ((s = upload(d, &gp, geo.data(), geo.size() * sizeof(P3Geo<T>))) != TF_OK) return s;
        d.geo2 = gp;
    }
    {
        std::vector<P3Dev<T>> dtv(1);
        P3Dev<T> &dt = dtv[0];
        for (int e = 0; e < 400; ++e) {
            dt.M[e] = (T)tab.M[e];
            for (int k = 0; k < 4; ++k) dt.C[k][e] = (T)tab.C[k][e];
        }
        for (int f = 0; f < 4; ++f) {
            for (int e = 0; e < 400; ++e) dt.FA[f][e] = T(0);
            for (int i = 0; i < 20; ++i)
                for (int c = 0; c < 12; ++c) dt.FU[f][i][c] = T(0);
            for (int r = 0; r < 10; ++r)
                for (int c = 0; c < 10; ++c) {
                    dt.FA[f][20 * tab.fn[f][r] + tab.fn[f][c]] = (T)tab.F[f][10 * r + c];
                    dt.FU[f][tab.fn[f][r]][c] = (T)tab.F[f][10 * r + c];
                }
        }
        P3Dev<T> *tp = nullptr;
        if ((s = upload(d, &tp, &dt, sizeof(dt))) != TF_OK) return s;
        d.p3tab = tp;
        int32_t fn[40];
        for (int f = 0; f < 4; ++f)
            for (int r = 0; r < 10; ++r) fn[10 * f + r] = tab.fn[f][r];
        if ((s = upload(d, &d.ho_pw, tab.p, sizeof(tab.p))) != TF_OK) return s;
        if ((s = upload(d, &d.ho_fn, fn, sizeof(fn))) != TF_OK) return s;
        if ((s = upload(d, &d.ho_fav, tab.fav[0], sizeof(tab.fav[0]))) != TF_OK) return s;
    }
    if ((s = upload_vec3<T>(d, &d.omega, p.quad->omega.data(), d.D, p.quad->w.data())) != TF_OK) return s;
    if ((s = upload(d, &d.mat, cell_material, sizeof(int32_t) * (size_t)d.C)) != TF_OK) return s;
    if ((s = upload(d, &d.sig_d, sigma_t, sizeof(double) * (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_t, sigma_t, (size_t)d.M * d.G)) != TF_OK) return s;
    if ((s = upload_typed<T>(d, &d.sigma_s, sigma_s, (size_t)d.M * d.G * d.G)) != TF_OK) return s;
    if ((s = upload(d, &d.vol, m.vol.data(), sizeof(double) * (size_t)d.C)) != TF_OK) return s;
    {
        std::vector<double> Qs((size_t)d.C * d.G * 20);
        for (int64_t c = 0; c < d.C; ++c)
            for (int gq = 0; gq < d.G; ++gq)
                for (int i = 0; i < 20; ++i) Qs[((size_t)c * 20 + i) * d.G + gq] = Q[((size_t)c * d.G + gq) * 20 + i];
        if ((s = upload_typed<T>(d, &d.Q, Qs.data(), Qs.size())) != TF_OK) return s;
    }
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
    if (cudaDeviceGetAttribute(&d.clock_khz, cudaDevAttrClockRate, d.device) != cudaSuccess) {
        d.clock_khz = 0;
        cudaGetLastError();
    }
    d.C = m.nc;
    d.nv = m.nv;
    d.G = p.G;
    d.D = p.quad->D;
    d.M = p.M;
    d.fp64 = p.opt.precision == TF_FP64;
    d.order = p.opt.order >= 2 ? p.opt.order : 1;
    d.hex = m.nf == 6;
    d.nb = d.hex ? 8 : d.order == 3 ? 20 : d.order == 2 ? 10 : 4;
    // pairing 0 = automatic: packed pairs unless G is a multiple of 32 (there the
    // shared-memory staged path is faster); 2 = packed pairs whenever G is even
    d.paired = d.order == 1 && !d.hex && !d.fp64 && d.G % 2 == 0 && (p.opt.pairing == 2 || (p.opt.pairing == 0 && d.G % 32 != 0)) &&
               g.cells_per_task <= 32 &&
               PairLayout(d.G, g.cells_per_task).bytes() <= 227u * 1024u;
    d.tsize = d.fp64 ? 8 : 4;
    const int64_t T = g.T();
    if ((uint64_t)g.down_list.size() >= (1ull << 32)) return fail(TF_ERR_ARG, "graph too large: 2^32 downwind edges");
    tf_status s;
    // task graph
    {
        // inflow masks of the task cell lists, caller face order -> sorted face order
        // (linear tetrahedra only)
        std::vector<uint8_t> remap(d.nodemajor() ? 0 : (size_t)m.nc * 16);
        for (int64_t c = 0; c < (d.nodemajor() ? 0 : m.nc); ++c) {
            int s2u[4];
            sorted_order(&m.tets[4 * c], s2u);
            for (uint32_t mk = 0; mk < 16; ++mk) {
                uint32_t r = 0;
                for (int j = 0; j < 4; ++j) r |= ((mk >> s2u[j]) & 1u) << j;
                remap[16 * c + mk] = (uint8_t)r;
            }
        }
        // (the higher orders and hexahedra keep the caller's face order)
        std::vector<uint32_t> cl(g.cell_list.size());
        for (size_t i = 0; i < cl.size(); ++i) {
            const uint32_t e = g.cell_list[i], c = e >> 4;
            cl[i] = d.nodemajor() ? e : (c << 4) | remap[16 * (size_t)c + (e & 15u)];
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
    if ((s = upload(d, &d.blevel, g.task_blevel.data(), (size_t)T * 4)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.counters, (size_t)T * 4)) != TF_OK) return s;
    // cell volumes / 4 (FP64) for the integrated flux
    {
        std::vector<double> v4(m.nc);
        for (int64_t c = 0; c < m.nc; ++c) v4[c] = 0.25 * m.vol[c];
        if ((s = upload(d, &d.vol4, v4.data(), v4.size() * 8)) != TF_OK) return s;
    }
    if (d.hex)
        s = d.fp64 ? create_typed_hex<double>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in)
                   : create_typed_hex<float>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in);
    else if (d.order == 3)
        s = d.fp64 ? create_typed_p3<double>(p, d, cell_material, sigma_t, sigma_s, Q)
                   : create_typed_p3<float>(p, d, cell_material, sigma_t, sigma_s, Q);
    else if (d.order == 2)
        s = d.fp64 ? create_typed_p2<double>(p, d, cell_material, sigma_t, sigma_s, Q)
                   : create_typed_p2<float>(p, d, cell_material, sigma_t, sigma_s, Q);
    else
        s = d.fp64 ? create_typed<double>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in)
                   : create_typed<float>(p, d, cell_material, sigma_t, sigma_s, Q, S1, psi_in);
    if (s != TF_OK) return s;
    if ((s = dmalloc(d, &d.q, (size_t)d.C * d.G * d.nb * d.tsize)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.phi_buf[0], (size_t)d.C * d.G * d.nb * 8)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.phi_buf[1], (size_t)d.C * d.G * d.nb * 8)) != TF_OK) return s;
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
    if ((s = dmalloc(d, &d.part, sizeof(double) * 6 * d.G * d.stats_blocks)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.leak, sizeof(double) * d.G)) != TF_OK) return s;
    TF_CUDA(cudaMemset(d.leak, 0, sizeof(double) * d.G));
    {
        std::vector<uint32_t> bc;
        for (int64_t c = 0; c < m.nc; ++c)
            for (int f = 0; f < m.nf; ++f)
                if (m.nbr[(int64_t)m.nf * c + f] < 0) {
                    bc.push_back((uint32_t)c);
                    break;
                }
        d.n_bcells = (int64_t)bc.size();
        if ((s = upload(d, &d.bcells, bc.data(), 4 * bc.size())) != TF_OK) return s;
    }
    if ((s = dmalloc(d, &d.gstats, sizeof(double) * 4 * d.G)) != TF_OK) return s;
    // direction chunks: as many directions per launch as the psi budget allows
    const size_t per_dir = (size_t)d.C * d.G * d.nb * d.tsize;
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
    // Bulk-synchronous schedules: per chunk, one bucket per (octant group, t-level),
    // groups in order and levels ascending within a group; a bucket lists the
    // tasks of all the group's directions on that level (direction, then block order).
    d.schedule = p.opt.schedule;
    if (d.schedule != TF_SCHED_AMT) {
        std::vector<uint32_t> order;
        order.reserve((size_t)T);
        d.bsp_bucket_host.clear();
        d.chunk_bucket_begin.assign(d.n_chunks + 1, 0);
        for (int k = 0; k < d.n_chunks; ++k) {
            const int a0 = k * Dc, a1 = std::min(d.D, a0 + Dc);
            const int ngrp = d.chunk_group_begin[k + 1] - d.chunk_group_begin[k];
            d.chunk_bucket_begin[k] = (int32_t)d.bsp_bucket_host.size();
            for (int j = 0; j < ngrp; ++j) {
                int L = 0;
                for (int a = a0; a < a1; ++a)
                    if (dir_group[a] == j) L = std::max(L, g.dir_levels[a]);
                std::vector<size_t> start(L + 1, 0);
                for (int a = a0; a < a1; ++a)
                    if (dir_group[a] == j)
                        for (int64_t t = g.dir_task_begin[a]; t < g.dir_task_begin[a + 1]; ++t) ++start[g.task_level[t] + 1];
                for (int l = 0; l < L; ++l) start[l + 1] += start[l];
                const size_t base = order.size();
                order.resize(base + start[L]);
                std::vector<size_t> pos(start.begin(), start.end() - 1);
                for (int a = a0; a < a1; ++a)
                    if (dir_group[a] == j)
                        for (int64_t t = g.dir_task_begin[a]; t < g.dir_task_begin[a + 1]; ++t)
                            order[base + pos[g.task_level[t]]++] = (uint32_t)t;
                for (int l = 0; l < L; ++l) d.bsp_bucket_host.push_back((uint32_t)(base + start[l]));
            }
        }
        d.chunk_bucket_begin[d.n_chunks] = (int32_t)d.bsp_bucket_host.size();
        d.bsp_bucket_host.push_back((uint32_t)order.size());
        // the claim counters of the buckets reuse the task counters: a bucket holds at least one task
        if ((int64_t)order.size() != T || (int64_t)d.bsp_bucket_host.size() - 1 > T)
            return fail(TF_ERR_DEVICE, "bulk-synchronous schedule does not cover the task graph");
        if ((s = upload(d, &d.bsp_order, order.data(), order.size() * 4)) != TF_OK) return s;
        if ((s = upload(d, &d.bsp_bucket, d.bsp_bucket_host.data(), d.bsp_bucket_host.size() * 4)) != TF_OK) return s;
        if ((s = dmalloc(d, &d.bsp_bar, sizeof(unsigned int))) != TF_OK) return s;
    }
    d.window = p.opt.octant_window > 0 ? p.opt.octant_window : 8;
    if ((s = upload(d, &d.dir_group, dir_group.data(), dir_group.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.group_total, group_total.data(), group_total.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.group_admit, group_admit.data(), group_admit.size() * 4)) != TF_OK) return s;
    if ((s = dmalloc(d, &d.group_rem, group_total.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.gseed, d.gseed_host.data(), d.gseed_host.size() * 4)) != TF_OK) return s;
    if ((s = upload(d, &d.seeds, seeds.data(), seeds.size() * 4)) != TF_OK) return s;
    d.seeds_host = seeds;
    if ((s = dmalloc(d, &d.slots, (size_t)d.max_chunk_tasks * 8)) != TF_OK) return s;
    TF_CUDA(cudaMemset(d.slots, 0, (size_t)d.max_chunk_tasks * 8));
    if ((s = dmalloc(d, &d.psi, per_dir * Dc)) != TF_OK) return s;
    // persistent grid: resident CTAs per SM x SMs
    d.wpc = p.opt.warps_per_cta > 0 ? std::min(p.opt.warps_per_cta, 4) : 4;  // launch bounds: 128 threads
    {
        // FP32 stages two cells per warp (six CTAs fit per SM), FP64 three; staging 2 / 3 force it
        const int ns = p.opt.staging == 3 ? 3 : p.opt.staging == 2 ? 2 : (d.fp64 ? 3 : 2);
        const size_t wb = d.fp64 ? staged_warp_bytes<double>(d.G, ns) : staged_warp_bytes<float>(d.G, ns);
        const size_t wb128 = (wb + 48 + 127) / 128 * 128;  // + the six mbarriers at the end
        d.staged = d.order == 1 && !d.hex && p.opt.staging != 1 && d.G % 32 == 0 && g.cells_per_task <= 64 &&
                   wb128 * d.wpc <= 227 * 1024;
        d.warp_smem = d.staged ? (uint32_t)wb128 : 0u;
        d.two_stage = d.staged && ns == 2 && !d.fp64;
    }
    // second order: staged in shared memory (FP32, G a multiple of 32, tasks of at most 32 cells)
    const bool p2_staged = d.order == 2 && !d.fp64 && d.G % 32 == 0 && g.cells_per_task <= 32 && p.opt.staging != 1 &&
                           ((p2_stage_bytes(d.G) * 2 + 48 + 127) / 128 * 128) * d.wpc <= 227 * 1024;
    if (p2_staged) d.warp_smem = (p2_stage_bytes(d.G) * 2 + 48 + 127) / 128 * 128;
    // third order: per warp the cell's group-independent matrix and the pivot rows, per CTA the tables
    if (d.order == 3) {
        d.warp_smem = ((d.fp64 ? p3_warp_bytes<double>() : p3_warp_bytes<float>()) + 127u) / 128u * 128u;
        d.cta_smem = d.fp64 ? sizeof(P3Dev<double>) : sizeof(P3Dev<float>);
    }
    // hexahedra: the group-independent matrices in shared memory once per cell when a batch of
    // 32 units touches at most five cells (G >= 8); staging = 1 keeps every lane on its own
    const bool hex_shared = d.hex && d.G >= 8 && p.opt.staging != 1;
    if (d.hex) d.warp_smem = hex_shared ? (hex_stage_bytes((int)d.tsize) + 127u) / 128u * 128u : 0u;
    d.mode = d.hex ? (hex_shared ? 9 : 8)
             : d.order == 3 ? 7
             : d.order == 2 ? (p2_staged ? 6 : 5)
             : d.paired  ? 3
             : d.staged  ? (d.two_stage ? 4 : 2)
                         : (d.G % 32 == 0 && g.cells_per_task <= 64 ? 1 : 0);
    // tasks whose cells depend on each other need a variant that solves a task's cells one
    // after another with every lane on the groups of one cell (modes 1, 2, 4)
    if (g.patches && !(d.mode == 1 || d.mode == 2 || d.mode == 4) )
        return fail(TF_ERR_ARG, "spatial-patch tasks need a kernel variant with lanes over one cell's groups");
    d.patches = g.patches;
    if (d.patches && (d.mode == 2 || d.mode == 4)) {
        // Per cell entry of a patch task, in the kernel's sorted face order (one byte):
        //   bits 0-2  upwind slots (interior inflow faces by rank) that the lanes fill, because
        //             the upwind cell is one of the task's NS - 1 cells listed just before: it is
        //             not solved yet when this cell's copies are issued;
        //   bit 3     the cell copies a row of an earlier cell of its own task (its lanes order
        //             their stores of that row before the copy);
        //   bits 4-5  slot + 1 of the next cell that takes this cell's solution (0: none);
        //   bits 6-7  the same for the cell after next (three stages).
        const int NS = d.mode == 4 ? 2 : 3;
        std::vector<uint8_t> aux(g.cell_list.size(), 0);
        std::vector<int32_t> pos_of;  // position in the current task, by cell (-1 outside)
        pos_of.assign(m.nc, -1);
        for (int64_t t = 0; t < T; ++t) {
            const uint32_t b = g.task_cell_begin[t], n = g.task_ncell[t];
            for (uint32_t i = 0; i < n; ++i) pos_of[g.cell_list[b + i] >> 4] = (int32_t)i;
            for (uint32_t i = 0; i < n; ++i) {
                const uint32_t e = g.cell_list[b + i], c = e >> 4, mk = e & 15u;
                int s2u[4];
                sorted_order(&m.tets[4 * (int64_t)c], s2u);
                int r = 0;
                for (int j = 0; j < 4; ++j) {
                    const int u = s2u[j];
                    const int32_t nb = m.nbr[4 * (int64_t)c + u];
                    if (!((mk >> u) & 1u) || nb < 0) continue;
                    const int32_t p = pos_of[nb];
                    if (p >= 0 && p < (int32_t)i) {
                        const int dist = (int)i - p;
                        if (dist <= NS - 1) {
                            aux[b + i] |= (uint8_t)(1u << r);
                            aux[b + p] |= (uint8_t)((r + 1) << (dist == 1 ? 4 : 6));
                        } else {
                            aux[b + i] |= 8u;
                        }
                    } else if (p >= (int32_t)i) {
                        return fail(TF_ERR_DEVICE, "patch task lists an upwind cell after its downwind cell");
                    }
                    ++r;
                }
            }
            for (uint32_t i = 0; i < n; ++i) pos_of[g.cell_list[b + i] >> 4] = -1;
        }
        if ((s = upload(d, &d.cells_aux, aux.data(), aux.size())) != TF_OK) return s;
    }
    if (d.paired) {
        d.staged = false;
        // three buffers unless two let more CTAs be resident per SM
        auto warp_bytes = [&](int ns) { return (PairLayout(d.G, g.cells_per_task, ns).bytes() + 48u + 127u) / 128u * 128u; };
        const uint32_t budget = 227u * 1024u;
        auto resident = [&](int ns) {
            const uint32_t w = warp_bytes(ns);
            if (w * d.wpc > budget) return 0;
            int n = 0;
            const void *k3 = (const void *)sweep_kernel<float, 3>;
            if (ensure_dyn_smem(k3, (int)(w * d.wpc)) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k3, 32 * d.wpc, (size_t)w * d.wpc) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            return n;
        };
        d.pair_stages = resident(2) > resident(3) ? 2 : 3;
        const uint32_t wb = warp_bytes(d.pair_stages);
        while (d.wpc > 1 && wb * d.wpc > budget) d.wpc /= 2;
        d.warp_smem = wb;
        const PairLayout L(d.G, g.cells_per_task, d.pair_stages);
        d.lpc_shift = (int)L.lpc_shift;
        d.ppl = (int)L.ppl;
    }
    if (d.nodemajor()) {
        // the node-major source update stages max(1, 256 / G) cells' flux in shared memory:
        // above 48 KB (large G) the kernel needs the opt-in limit
        const size_t smem2 = (size_t)std::max(1, 256 / d.G) * d.G * d.nb * d.tsize;
        const void *sfn = d.nb == 8    ? (d.fp64 ? (const void *)source_ho_kernel<double, 8> : (const void *)source_ho_kernel<float, 8>)
                          : d.nb == 20 ? (d.fp64 ? (const void *)source_ho_kernel<double, 20> : (const void *)source_ho_kernel<float, 20>)
                                       : (d.fp64 ? (const void *)source_ho_kernel<double, 10> : (const void *)source_ho_kernel<float, 10>);
        if (smem2 > 48 * 1024) TF_CUDA(ensure_dyn_smem(sfn, (int)smem2));
    }
    const int dyn = (int)(d.warp_smem * d.wpc + d.cta_smem);
    const void *kfn = d.mode == 9   ? (d.fp64 ? (const void *)sweep_kernel<double, 9> : (const void *)sweep_kernel<float, 9>)
                      : d.mode == 8 ? (d.fp64 ? (const void *)sweep_kernel<double, 8> : (const void *)sweep_kernel<float, 8>)
                      : d.mode == 7 ? (d.fp64 ? (const void *)sweep_kernel<double, 7> : (const void *)sweep_kernel<float, 7>)
                      : d.mode == 6 ? (const void *)sweep_kernel<float, 6>
                      : d.mode == 5 ? (d.fp64 ? (const void *)sweep_kernel<double, 5> : (const void *)sweep_kernel<float, 5>)
                      : d.fp64 ? (d.mode == 2 ? (const void *)sweep_kernel<double, 2>
                                            : d.mode == 1 ? (const void *)sweep_kernel<double, 1> : (const void *)sweep_kernel<double, 0>)
                             : (d.mode == 3   ? (const void *)sweep_kernel<float, 3>
                                : d.mode == 4 ? (const void *)sweep_kernel<float, 4>
                                : d.mode == 2 ? (const void *)sweep_kernel<float, 2>
                                : d.mode == 1 ? (const void *)sweep_kernel<float, 1>
                                              : (const void *)sweep_kernel<float, 0>);
    if (dyn > 0) TF_CUDA(ensure_dyn_smem(kfn, dyn));
    int per_sm = 0;
    TF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * d.wpc, dyn));
    if (p.opt.ctas_per_sm > 0) per_sm = std::min(per_sm, p.opt.ctas_per_sm);
    d.grid = std::max(1, per_sm) * d.sm_count;
    if (d.schedule != TF_SCHED_AMT) {
        // bulk-synchronous kernel of the same variant; its cooperative launch needs a co-resident grid
        const void *bfn = d.fp64 ? bsp_kernel_fn<double>(d.mode) : bsp_kernel_fn<float>(d.mode);
        if (dyn > 0) TF_CUDA(ensure_dyn_smem(bfn, dyn));
        int bsm = 0;
        TF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bsm, bfn, 32 * d.wpc, dyn));
        if (p.opt.ctas_per_sm > 0) bsm = std::min(bsm, p.opt.ctas_per_sm);
        if (bsm < 1) return fail(TF_ERR_CUDA, "bulk-synchronous sweep kernel cannot be resident");
        d.bsp_grid = bsm * d.sm_count;
        p.stats.n_buckets = d.chunk_bucket_begin[d.n_chunks];
    }
    d.ev_start.resize(1 + 2 * d.n_chunks);
    d.ev_stop.resize(1 + 2 * d.n_chunks);
    for (size_t i = 0; i < d.ev_start.size(); ++i) {
        TF_CUDA(cudaEventCreate(&d.ev_start[i]));
        TF_CUDA(cudaEventCreate(&d.ev_stop[i]));
    }
    TF_CUDA(cudaDeviceSynchronize());
    // source; per chunk: begin, fill, sweep, end, phi and (with boundary cells) leakage
    if (d.schedule == TF_SCHED_AMT)
        p.stats.launches_per_step = 1 + (5 + (d.n_bcells > 0 ? 1 : 0)) * (int64_t)d.n_chunks;
    else  // begin, sweep (one, or one per bucket), end, phi, leakage
        p.stats.launches_per_step = 1 + (3 + (d.n_bcells > 0 ? 1 : 0)) * (int64_t)d.n_chunks +
                                    (d.schedule == TF_SCHED_BSP ? (int64_t)d.n_chunks : (int64_t)p.stats.n_buckets);
    p.stats.kernel_mode = d.mode;
    TF_CUDA(cudaStreamCreateWithFlags(&d.istream, cudaStreamNonBlocking));
    TF_CUDA(cudaEventCreateWithFlags(&d.ev_user, cudaEventDisableTiming));
    TF_CUDA(cudaEventCreateWithFlags(&d.ev_done, cudaEventDisableTiming));
    p.stats.n_tasks = T;
    p.stats.n_units = (int64_t)d.C * d.D * d.G;
    p.stats.n_dirs = d.D;
    p.stats.max_level = g.max_level;
    p.stats.n_chunks = d.n_chunks;
    p.stats.grid_ctas = d.schedule == TF_SCHED_AMT ? d.grid : d.bsp_grid;
    p.stats.warps_per_cta = d.wpc;
    p.stats.cells_per_task = g.cells_per_task;
    p.stats.task_shape = g.patches ? TF_TASK_PATCHES : TF_TASK_LEVELS;
    p.stats.lagged_faces = g.n_lagged();
    if (g.n_lagged() > 0) {
        // lag words and slots; the lag buffer starts at zero (the first step's lagged faces see
        // no inflow from the previous step)
        d.n_lag = g.n_lagged();
        d.lag_dir_begin = g.lag_dir_begin;
        if ((s = upload(d, &d.lagw, g.cell_lag.data(), g.cell_lag.size() * 4)) != TF_OK) return s;
        if ((s = upload(d, &d.lag_slots, g.lag_slots.data(), g.lag_slots.size() * 4)) != TF_OK) return s;
        const size_t lb = (size_t)d.n_lag * 4 * d.G * d.tsize;
        if ((s = dmalloc(d, &d.lagbuf, lb)) != TF_OK) return s;
        TF_CUDA(cudaMemset(d.lagbuf, 0, lb));
    }
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
    for (cudaGraphExec_t g : d->gexec)
        if (g) cudaGraphExecDestroy(g);
    if (d->ev_user) cudaEventDestroy(d->ev_user);
    if (d->ev_done) cudaEventDestroy(d->ev_done);
    if (d->istream) cudaStreamDestroy(d->istream);
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

// Device address of page-locked host memory mapped into the device's address space
// (cudaHostAlloc / torch pin_memory); NULL for anything else.
void *mapped_host_pointer(const void *ptr)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// q <- source(phi_in), for one problem.
template <class T> void launch_source(Problem &p, const double *phi_in, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    if (d.nodemajor()) {
        const int cpc2 = std::max(1, 256 / d.G);
        const size_t smem2 = (size_t)cpc2 * d.G * d.nb * sizeof(T);
        const int blocks2 = (int)std::min<int64_t>((d.C + cpc2 - 1) / cpc2, (int64_t)d.sm_count * 16);
        if (d.hex)
            source_ho_kernel<T, 8><<<blocks2, 256, smem2, st>>>(phi_in, (const T *)d.Q, (const T *)d.sigma_s, d.mat,
                                                                (T *)d.q, d.C, d.G, cpc2);
        else if (d.order == 3)
            source_ho_kernel<T, 20><<<blocks2, 256, smem2, st>>>(phi_in, (const T *)d.Q, (const T *)d.sigma_s, d.mat,
                                                                 (T *)d.q, d.C, d.G, cpc2);
        else
            source_ho_kernel<T, 10><<<blocks2, 256, smem2, st>>>(phi_in, (const T *)d.Q, (const T *)d.sigma_s, d.mat,
                                                                 (T *)d.q, d.C, d.G, cpc2);
        cudaMemsetAsync(d.leak, 0, sizeof(double) * d.G, st);
        return;
    }
    const int cpc = std::max(1, 256 / d.G);
    const size_t smem = (size_t)cpc * d.G * 4 * sizeof(T);
    const int blocks = (int)std::min<int64_t>((d.C + cpc - 1) / cpc, (int64_t)d.sm_count * 16);
    source_kernel<T><<<blocks, 256, smem, st>>>(phi_in, (const V4<T> *)d.Q, (const T *)d.sigma_s,
                                                (const CellGeo<T> *)d.geo, (V4<T> *)d.q, d.C, d.G, cpc,
                                                d.paired ? 1 : 0);
    cudaMemsetAsync(d.leak, 0, sizeof(double) * d.G, st);  // the phi kernels add this step's leakage
}

// Statistics, balance and stopping test of a higher-order iterate (NB nodes per cell).
template <int NB> void launch_stats_ho(Problem &p, const double *cur, const double *nxt, bool res, BalIn bi,
                                       cudaStream_t st)
{
    DeviceState &d = *p.dev;
    const dim3 blk(32, 8);
    const double *pwc = d.hex_pw;  // hexahedra: per-cell weights; else V_c times the element's
    if (d.fp64) {
        if (res) stats_ho_kernel<double, true, NB><<<d.stats_blocks, blk, 0, st>>>(nxt, cur, d.vol, d.C, d.G, d.part, bi, d.ho_pw, pwc);
        else stats_ho_kernel<double, false, NB><<<d.stats_blocks, blk, 0, st>>>(nxt, cur, d.vol, d.C, d.G, d.part, bi, d.ho_pw, pwc);
    } else {
        if (res) stats_ho_kernel<float, true, NB><<<d.stats_blocks, blk, 0, st>>>(nxt, cur, d.vol, d.C, d.G, d.part, bi, d.ho_pw, pwc);
        else stats_ho_kernel<float, false, NB><<<d.stats_blocks, blk, 0, st>>>(nxt, cur, d.vol, d.C, d.G, d.part, bi, d.ho_pw, pwc);
    }
    if (res) {
        finish_stats_res_kernel<<<(d.G + 127) / 128, 128, 0, st>>>(d.part, d.stats_blocks, d.G, d.gstats, d.leak, d.ctrl);
    } else {
        finish_stats_kernel<<<(d.G + 127) / 128, 128, 0, st>>>(d.part, d.stats_blocks, d.G, d.gstats, d.leak, d.ctrl);
        residual_ho_kernel<NB><<<d.stats_blocks, blk, 0, st>>>(nxt, cur, d.gstats, d.C, d.G, p.opt.residual_floor, d.ctrl);
    }
}

// Statistics, particle balance and stopping test of the iterate nxt (previous: cur).
void launch_stats(Problem &p, const double *cur, const double *nxt, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    BalIn bi;
    bi.mat = d.mat;
    bi.sig = d.sig_d;
    bi.q = d.q;
    bi.qmode = d.paired ? 2 : (d.fp64 ? 1 : 0);
    bi.leak = d.leak;
    cudaMemsetAsync(&d.ctrl->residual_bits, 0, 16, st);  // residual_bits, balance_bits
    if (d.nodemajor()) {
        const bool res = p.opt.residual_floor >= 1.0;
        if (d.hex) launch_stats_ho<8>(p, cur, nxt, res, bi, st);
        else if (d.order == 3) launch_stats_ho<20>(p, cur, nxt, res, bi, st);
        else launch_stats_ho<10>(p, cur, nxt, res, bi, st);
        return;
    }
    if (p.opt.residual_floor >= 1.0) {
        stats_res_kernel<<<d.stats_blocks, dim3(32, 8), 0, st>>>(nxt, cur, d.vol4, d.C, d.G, d.part, bi);
        finish_stats_res_kernel<<<(d.G + 127) / 128, 128, 0, st>>>(d.part, d.stats_blocks, d.G, d.gstats, d.leak,
                                                                   d.ctrl);
    } else {
        stats_kernel<<<d.stats_blocks, dim3(32, 8), 0, st>>>(nxt, d.vol4, d.C, d.G, d.part, bi);
        finish_stats_kernel<<<(d.G + 127) / 128, 128, 0, st>>>(d.part, d.stats_blocks, d.G, d.gstats, d.leak, d.ctrl);
        residual_kernel<<<d.stats_blocks, dim3(32, 8), 0, st>>>(nxt, cur, d.gstats, d.C, d.G, p.opt.residual_floor,
                                                                d.ctrl);
    }
}

// Sweep arguments of direction chunk k of one problem (queue fields for a launch of its own).
// Lagged back edges: after a chunk's sweep, the upwind values each lagged face of the chunk's
// directions will read in the next transport step (thread per slot, face-local node, group).
template <class T>
__global__ void lag_gather_kernel(const uint32_t *__restrict__ slots, int64_t s0, int64_t s1,
                                  const HexGeo<T> *__restrict__ geo, const T *__restrict__ psi, int dir_begin, int64_t C,
                                  int G, T *__restrict__ lagbuf)
{
    const int64_t n = (s1 - s0) * 4 * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + i / (4 * G);
        const int l = (int)((i / G) % 4), g = (int)(i % G);
        const uint32_t a = slots[2 * s], cf = slots[2 * s + 1];
        const uint32_t c = cf >> 3, f = cf & 7u;
        const int32_t nb = geo[c].nbr[f];
        const uint32_t node = (geo[c].nmap[f] >> (4 * l)) & 15u;
        lagbuf[(s * 4 + l) * G + g] = psi[(((int64_t)a - dir_begin) * C + nb) * 8 * G + (int64_t)node * G + g];
    }
}

template <class T> void launch_lag_gather(Problem &p, int k, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    if (d.n_lag == 0) return;
    const int a0 = k * d.Dc, a1 = std::min(d.D, a0 + d.Dc);
    const int64_t s0 = d.lag_dir_begin[a0], s1 = d.lag_dir_begin[a1];
    if (s1 <= s0) return;
    const int64_t n = (s1 - s0) * 4 * d.G;
    const int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)d.sm_count * 8);
    lag_gather_kernel<T><<<nb, 256, 0, st>>>(d.lag_slots, s0, s1, (const HexGeo<T> *)d.geo2, (const T *)d.psi, a0,
                                             d.C, d.G, (T *)d.lagbuf);
}

template <class T> SweepArgs<T> make_args(Problem &p, int k)
{
    DeviceState &d = *p.dev;
    const int64_t t0 = d.chunk_task_begin[k], t1 = d.chunk_task_begin[k + 1];
    const int a0 = k * d.Dc;
    const int gb = d.chunk_group_begin[k], ng = d.chunk_group_begin[k + 1] - gb;
    SweepArgs<T> A;
    std::memset(&A, 0, sizeof(A));
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
    A.hexv = d.hexv;
    A.lagw = d.lagw;
    A.lagbuf = (const T *)d.lagbuf;
    A.C = d.C;
    A.G = d.G;
    A.dir_begin = a0;
    A.task_begin = (uint32_t)t0;
    A.task_end = (uint32_t)t1;
    A.n_tasks = (unsigned long long)(t1 - t0);
    A.wait_limit_ns = (unsigned long long)(p.opt.wait_limit_s * 1e9);
    A.max_cells = p.graph.cells_per_task;
    A.intra = d.patches ? 1 : 0;
    A.blevel = p.opt.task_order == 1 ? nullptr : d.blevel;

    A.aux = d.cells_aux;
    A.warp_smem = d.warp_smem;
    A.dir_group = d.dir_group;
    A.group_rem = d.group_rem + gb;
    A.group_admit = d.group_admit + gb;
    A.gseed = d.gseed + gb + k;
    A.seeds = d.seeds;
    A.n_groups = ng;
    A.window = std::min(d.window, ng);
    A.lpc_shift = d.lpc_shift;
    A.ppl = d.ppl;
    A.stages = d.pair_stages;
    A.mode = d.mode;
    A.geo2 = d.geo2;
    A.p3tab = d.p3tab;
    A.keep_max = p.opt.keep_ready > 0 ? std::min(p.opt.keep_ready, 4) : 1;
    return A;
}

// phi_out (+)= sum over chunk k's directions of w_a psi_a, for one problem.
template <class T> void launch_phi(Problem &p, int k, double *phi_out, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    const size_t CG = (size_t)d.C * d.G;
    const int a0 = k * d.Dc, a1 = std::min(d.D, a0 + d.Dc);
    const int pb = (int)std::min<size_t>((CG + 255) / 256, (size_t)d.sm_count * 32);
    if (d.nodemajor()) {
        const bool pair = !d.fp64 && p.opt.phi_accumulate == TF_PHI_PAIR;
        const T *ps = (const T *)d.psi;
        if (d.hex) {
            if (pair) phi_ho_kernel<T, true, 8><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
            else phi_ho_kernel<T, false, 8><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
        } else if (d.order == 3) {
            if (pair) phi_ho_kernel<T, true, 20><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
            else phi_ho_kernel<T, false, 20><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
        } else {
            if (pair) phi_ho_kernel<T, true, 10><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
            else phi_ho_kernel<T, false, 10><<<pb, 256, 0, st>>>(ps, d.wts + a0, a1 - a0, d.C, d.G, phi_out, k > 0);
        }
        if (d.n_bcells > 0) {
            const int lb = (int)std::min<int64_t>((d.n_bcells * d.G + 255) / 256, (int64_t)d.sm_count * 16);
            const HoTables tb{d.ho_pw, d.ho_fn, d.ho_fav};
            const V4<T> *om = (const V4<T> *)d.omega + a0;
            if (d.hex)
                leak_hex_kernel<T><<<lb, 256, 0, st>>>(ps, d.wts + a0, om, a1 - a0, d.C, d.G, d.bcells, d.n_bcells,
                                                       (const HexGeo<T> *)d.geo2, d.hexv, (const T *)d.psi_in, d.leak);
            else if (d.order == 3)
                leak_ho_kernel<T, 20, 10, P3Geo<T>><<<lb, 256, 0, st>>>(ps, d.wts + a0, om, a1 - a0, d.C, d.G, d.bcells,
                                                                        d.n_bcells, (const P3Geo<T> *)d.geo2, tb, d.leak);
            else
                leak_ho_kernel<T, 10, 6, P2Geo<T>><<<lb, 256, 0, st>>>(ps, d.wts + a0, om, a1 - a0, d.C, d.G, d.bcells,
                                                                       d.n_bcells, (const P2Geo<T> *)d.geo2, tb, d.leak);
        }
        return;
    }
    if (d.paired) {
        const size_t CP = CG / 2;
        const int pb2 = (int)std::min<size_t>((CP + 255) / 256, (size_t)d.sm_count * 32);
        if (p.opt.phi_accumulate == TF_PHI_PAIR)
            phi_pair_kernel<true><<<pb2, 256, 0, st>>>((const float *)d.psi, d.wts + a0, a1 - a0, CP, d.G,
                                                       (const CellGeo<float> *)d.geo, phi_out, k > 0);
        else
            phi_pair_kernel<false><<<pb2, 256, 0, st>>>((const float *)d.psi, d.wts + a0, a1 - a0, CP, d.G,
                                                        (const CellGeo<float> *)d.geo, phi_out, k > 0);
    } else if (!d.fp64 && p.opt.phi_accumulate == TF_PHI_PAIR) {
        phi_kernel<T, true><<<pb, 256, 0, st>>>((const V4<T> *)d.psi, d.wts + a0, a1 - a0, CG, d.G,
                                                (const CellGeo<T> *)d.geo, phi_out, k > 0);
    } else {
        phi_kernel<T, false><<<pb, 256, 0, st>>>((const V4<T> *)d.psi, d.wts + a0, a1 - a0, CG, d.G,
                                                 (const CellGeo<T> *)d.geo, phi_out, k > 0);
    }
    // boundary leakage of this chunk's directions (particle balance)
    if (d.n_bcells > 0) {
        const int lb = (int)std::min<int64_t>((d.n_bcells * d.G + 255) / 256, (int64_t)d.sm_count * 16);
        if (d.paired)
            leak_kernel<float, true><<<lb, 256, 0, st>>>((const float *)d.psi, d.wts + a0, (const float4 *)d.omega + a0,
                                                         a1 - a0, d.C, d.G, d.bcells, d.n_bcells,
                                                         (const CellGeo<float> *)d.geo, d.tets,
                                                         (const float *)d.psi_in, d.leak);
        else
            leak_kernel<T, false><<<lb, 256, 0, st>>>((const T *)d.psi, d.wts + a0, (const V4<T> *)d.omega + a0, a1 - a0,
                                                      d.C, d.G, d.bcells, d.n_bcells, (const CellGeo<T> *)d.geo,
                                                      d.tets, (const T *)d.psi_in, d.leak);
    }
}

template <class T> tf_status launch_step(Problem &p, const double *phi_in, double *phi_out, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    TF_CUDA(record_event(d.ev_start[0], st));
    launch_source<T>(p, phi_in, st);
    TF_CUDA(cudaGetLastError());
    TF_CUDA(record_event(d.ev_stop[0], st));
    for (int k = 0; k < d.n_chunks; ++k) {
        if (d.schedule != TF_SCHED_AMT) {
            // bulk-synchronous: the chunk's buckets in sequence, a barrier after each
            begin_kernel<<<1, 1, 0, st>>>(d.ctrl, 0ull, k == 0, 0);
            const int b0 = d.chunk_bucket_begin[k], b1 = d.chunk_bucket_begin[k + 1];
            TF_CUDA(cudaMemsetAsync(d.counters + b0, 0, sizeof(int) * (size_t)(b1 - b0), st));
            TF_CUDA(cudaMemsetAsync(d.bsp_bar, 0, sizeof(unsigned int), st));
            const SweepArgs<T> A = make_args<T>(p, k);
            BspArgs S{d.bsp_order, d.bsp_bucket, d.counters, d.bsp_bar, b0, b1, p.opt.inject_stall ? 1 : 0};
            const size_t dyn = (size_t)d.warp_smem * d.wpc + d.cta_smem;
            TF_CUDA(record_event(d.ev_start[1 + 2 * k], st));
            if (d.schedule == TF_SCHED_BSP) {
                TF_CUDA(launch_bsp<T>(A, S, d.mode, d.bsp_grid, 32 * d.wpc, dyn, true, st));
            } else {
                for (int b = b0; b < b1; ++b) {
                    S.b_lo = b;
                    S.b_hi = b + 1;
                    const int64_t nt = (int64_t)d.bsp_bucket_host[b + 1] - (int64_t)d.bsp_bucket_host[b];
                    const int gr = (int)std::min<int64_t>(d.bsp_grid, (nt + d.wpc - 1) / d.wpc);
                    TF_CUDA(launch_bsp<T>(A, S, d.mode, gr, 32 * d.wpc, dyn, false, st));
                }
            }
            TF_CUDA(record_event(d.ev_stop[1 + 2 * k], st));
            end_kernel<<<1, 1, 0, st>>>(d.ctrl);
            launch_lag_gather<T>(p, k, st);
            TF_CUDA(record_event(d.ev_start[2 + 2 * k], st));
            launch_phi<T>(p, k, phi_out, st);
            TF_CUDA(cudaGetLastError());
            TF_CUDA(record_event(d.ev_stop[2 + 2 * k], st));
            d.last_chunk = k;
            continue;
        }
        const int64_t t0 = d.chunk_task_begin[k], t1 = d.chunk_task_begin[k + 1];
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
        const SweepArgs<T> A = make_args<T>(p, k);
        TF_CUDA(record_event(d.ev_start[1 + 2 * k], st));
        const size_t dyn = (size_t)d.warp_smem * d.wpc + d.cta_smem;
        if constexpr (sizeof(T) == 4) {
            if (d.mode == 3) sweep_kernel<T, 3><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
            if (d.mode == 4) sweep_kernel<T, 4><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
            if (d.mode == 6) sweep_kernel<T, 6><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        }
        if (d.mode == 3 || d.mode == 4 || d.mode == 6) {
        } else if (d.mode == 9)
            sweep_kernel<T, 9><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        else if (d.mode == 8)
            sweep_kernel<T, 8><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        else if (d.mode == 7)
            sweep_kernel<T, 7><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        else if (d.mode == 5)
            sweep_kernel<T, 5><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        else if (d.mode == 2)
            sweep_kernel<T, 2><<<d.grid, 32 * d.wpc, dyn, st>>>(A);
        else if (d.mode == 1)
            sweep_kernel<T, 1><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        else
            sweep_kernel<T, 0><<<d.grid, 32 * d.wpc, 0, st>>>(A);
        TF_CUDA(cudaGetLastError());
        TF_CUDA(record_event(d.ev_stop[1 + 2 * k], st));
        end_kernel<<<1, 1, 0, st>>>(d.ctrl);
        launch_lag_gather<T>(p, k, st);
        TF_CUDA(record_event(d.ev_start[2 + 2 * k], st));
        launch_phi<T>(p, k, phi_out, st);
        TF_CUDA(cudaGetLastError());
        TF_CUDA(record_event(d.ev_stop[2 + 2 * k], st));
        d.last_chunk = k;
    }
    return TF_OK;
}

tf_status step(Problem &p, const double *phi_in, double *phi_out, cudaStream_t st)
{
    return p.dev->fp64 ? launch_step<double>(p, phi_in, phi_out, st) : launch_step<float>(p, phi_in, phi_out, st);
}

// Reads the control block after the stream drained; turns a device error into a status.
tf_status collect(Problem &p, cudaStream_t st, bool copied = false)
{
    DeviceState &d = *p.dev;
    if (!copied) TF_CUDA(cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    TF_CUDA(cudaStreamSynchronize(st));
    const Ctrl &c = *d.ctrl_host;
    tf_stats &s = p.stats;
    s.tasks_executed = (int64_t)c.tasks_done;
    s.wait_polls = (int64_t)c.polls;
    s.wait_seconds = c.wait_ns * 1e-9;
    s.busy_seconds = c.busy_ns * 1e-9;
    s.kernel_seconds = c.kernel_ns * 1e-9;
    s.mean_ready = c.pops ? (double)c.depth_sum / (double)c.pops : 0.0;
    s.data_wait_seconds = d.clock_khz > 0 ? (double)c.data_wait_cycles / (1e3 * d.clock_khz) : 0.0;
    {
        // CUDA-event times of the step's kernels (events recorded as external
        // nodes when the step runs inside a captured graph)
        float ms = 0.f;
        double src = 0.0, sw = 0.0, ph = 0.0;
        bool ok = cudaEventElapsedTime(&ms, d.ev_start[0], d.ev_stop[0]) == cudaSuccess;
        src = ms * 1e-3;
        for (int k = 0; ok && k < d.n_chunks; ++k) {
            ok = cudaEventElapsedTime(&ms, d.ev_start[1 + 2 * k], d.ev_stop[1 + 2 * k]) == cudaSuccess;
            sw += ms * 1e-3;
            ok = ok && cudaEventElapsedTime(&ms, d.ev_start[2 + 2 * k], d.ev_stop[2 + 2 * k]) == cudaSuccess;
            ph += ms * 1e-3;
        }
        if (ok) {
            s.source_event_seconds = src;
            s.sweep_event_seconds = sw;
            s.phi_event_seconds = ph;
            s.cum_source_event_seconds += src;
            s.cum_sweep_event_seconds += sw;
            s.cum_phi_event_seconds += ph;
            s.cum_steps += 1;
        } else {
            cudaGetLastError();
        }
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

// Direction sharding: the partners' sum of a partial buffer (phi, or the leakage per group).
static tf_status reduce_partial(Problem &p, double *buf, int64_t count, cudaStream_t st)
{
    const int32_t r = p.reduce(p.reduce_user, buf, count, (void *)st);
    if (r != 0) return fail(TF_ERR_CUDA, "reduce callback returned " + std::to_string(r));
    TF_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status device_sweep(Problem &p, const double *phi_in, double *phi_out, void *stream)
{
    DeviceState &d = *p.dev;
    TF_CUDA(cudaSetDevice(d.device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)d.C * d.G * d.nb * 8;
    const double *in = phi_in;
    double *out = phi_out;
    // Pinned, mapped host buffers are read by the source kernel and written by the phi
    // kernel directly (over the host link, overlapped with their work); other host
    // memory goes through copies to and from device buffers.
    const bool host_in = !is_device_pointer(phi_in), host_out = !is_device_pointer(phi_out);
    const double *map_in = host_in ? (const double *)mapped_host_pointer(phi_in) : nullptr;
    double *map_out = host_out ? (double *)mapped_host_pointer(phi_out) : nullptr;
    if (host_in) {
        if (map_in) {
            in = map_in;
        } else {
            TF_CUDA(cudaMemcpyAsync(d.phi_buf[0], phi_in, bytes, cudaMemcpyHostToDevice, st));
            in = d.phi_buf[0];
        }
    }
    if (p.reduce) map_out = nullptr;  // the partners' sum works on a device buffer
    if (host_out) out = map_out ? map_out : d.phi_buf[1];
    tf_status s = step(p, in, out, st);
    if (s != TF_OK) return s;
    if (p.reduce && (s = reduce_partial(p, out, (int64_t)(bytes / 8), st)) != TF_OK) return s;
    if (host_out && !map_out) TF_CUDA(cudaMemcpyAsync(phi_out, out, bytes, cudaMemcpyDeviceToHost, st));
    return collect(p, st);
}

namespace {

// One source iteration cur -> nxt: transport step, FP64 statistics and
// stopping test, and the control block copied to pinned host memory.
tf_status enqueue_iteration(Problem &p, const double *cur, double *nxt, cudaStream_t st)
{
    DeviceState &d = *p.dev;
    tf_status s = step(p, cur, nxt, st);
    if (s != TF_OK) return s;
    if (p.reduce) {  // direction sharding: every partner continues from the full phi and leakage
        if ((s = reduce_partial(p, nxt, (int64_t)d.C * d.G * d.nb, st)) != TF_OK) return s;
        if ((s = reduce_partial(p, d.leak, d.G, st)) != TF_OK) return s;
    }
    launch_stats(p, cur, nxt, st);
    TF_CUDA(cudaGetLastError());
    TF_CUDA(cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    return TF_OK;
}

// Captures the two ping-pong iterations as CUDA graphs on the internal stream.
// Returns false (and leaves gexec empty) if capture is not possible.
bool build_iteration_graphs(Problem &p)
{
    DeviceState &d = *p.dev;
    d.graphs_tried = true;
    for (int k = 0; k < 2; ++k) {
        double *cur = d.phi_buf[k], *nxt = d.phi_buf[1 - k];
        if (cudaStreamBeginCapture(d.istream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
        const tf_status s = enqueue_iteration(p, cur, nxt, d.istream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(d.istream, &g);
        if (s != TF_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            break;
        }
        const cudaError_t ei = cudaGraphInstantiate(&d.gexec[k], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            d.gexec[k] = nullptr;
            break;
        }
    }
    if (!d.gexec[0] || !d.gexec[1]) {
        for (auto &g : d.gexec)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace

// Source iteration on the problem's internal stream, ordered after the
// caller's stream and before the return.  Each iteration is one launch of a
// captured CUDA graph (direct launches if capture is unavailable), followed by
// a read of the control block (residual, device errors) from pinned memory.
tf_status device_iterate(Problem &p, double tol, int32_t max_iters, double *phi, tf_iter_info *info, void *stream)
{
    DeviceState &d = *p.dev;
    TF_CUDA(cudaSetDevice(d.device));
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t st = d.istream;
    const size_t CG = (size_t)d.C * d.G;
    const size_t bytes = CG * d.nb * 8;
    const bool host = !is_device_pointer(phi);
    TF_CUDA(cudaEventRecord(d.ev_user, user));
    TF_CUDA(cudaStreamWaitEvent(st, d.ev_user, 0));
    if (!d.graphs_tried && !p.reduce) build_iteration_graphs(p);
    int k = 0;  // phi_buf[k] holds the current iterate
    TF_CUDA(cudaMemcpyAsync(d.phi_buf[0], phi, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    double r = INFINITY, bal = 0.0;
    int it = 0;
    bool conv = false;
    for (it = 1; it <= max_iters; ++it) {
        if (d.gexec[k] && !p.reduce) {
            TF_CUDA(cudaGraphLaunch(d.gexec[k], st));
        } else {
            const tf_status s = enqueue_iteration(p, d.phi_buf[k], d.phi_buf[1 - k], st);
            if (s != TF_OK) return s;
        }
        d.last_chunk = d.n_chunks - 1;
        const tf_status s = collect(p, st, true);
        if (s != TF_OK) return s;
        std::memcpy(&r, &d.ctrl_host->residual_bits, sizeof(double));
        std::memcpy(&bal, &d.ctrl_host->balance_bits, sizeof(double));
        if (info && info->residual_history) info->residual_history[it - 1] = r;
        k = 1 - k;
        if (r < tol) {
            conv = true;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    // integrated flux of the final phi (already in gstats for the last iterate)
    TF_CUDA(cudaMemcpyAsync(d.gstats_host, d.gstats, sizeof(double) * 4 * d.G, cudaMemcpyDeviceToHost, st));
    TF_CUDA(cudaMemcpyAsync(phi, d.phi_buf[k], bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    TF_CUDA(cudaEventRecord(d.ev_done, st));
    TF_CUDA(cudaStreamWaitEvent(user, d.ev_done, 0));
    TF_CUDA(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = it;
        info->converged = conv ? 1 : 0;
        info->residual = r;
        info->balance = bal;
        double tot = 0.0;
        for (int g = 0; g < d.G; ++g) {
            tot += d.gstats_host[4 * g + 1];
            if (info->integrated_flux) info->integrated_flux[g] = d.gstats_host[4 * g + 1];
        }
        info->integrated_total = tot;
    }
    return conv ? TF_OK : fail(TF_ERR_NOT_CONVERGED, "source iteration reached max_iters");
}


// ================================================================ batched problems
// Independent problems (meshes, direction sets, group counts of their own, one
// precision) swept together: for each direction-chunk index c, one persistent
// launch of sweep_batch_kernel runs the chunk-c tasks of every problem through
// one shared ticket queue.  Source updates, phi reductions and statistics stay
// per problem.  Each source iteration is a captured CUDA graph (one per
// ping-pong parity) for the current set of unconverged problems; the graphs
// are captured again when a problem converges and leaves the set.
namespace {

__global__ void batch_seed_kernel(const Ctrl *ctrl, unsigned long long *slots, const uint32_t *seeds, uint32_t n)
{
    const unsigned epoch = ctrl->epoch;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        slots[i] = ((unsigned long long)epoch << 32) | seeds[i];
}

struct BatchRun {
    std::vector<Problem *> P;
    int device = 0, n = 0, max_chunks = 0, sm_count = 0;
    bool fp64 = false;
    bool hex = false;  // the batch holds hexahedral problems
    Ctrl *ctrl = nullptr, *ctrl_host = nullptr;
    unsigned long long *slots = nullptr;
    void *args = nullptr;          // [max_chunks][n] SweepArgs<T>
    uint32_t *offsets = nullptr;   // [max_chunks][n + 1]
    uint32_t *seeds = nullptr;     // [max_chunks][seed_cap]
    size_t seed_cap = 0, task_cap = 0;
    std::vector<std::vector<int>> part;  // per chunk: participating problems of the active set
    std::vector<uint64_t> n_tasks, n_seeds;
    int grid = 0, wpc = 4;
    uint32_t warp_smem = 48;
    cudaStream_t st = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    ~BatchRun()
    {
        for (auto &g : gexec)
            if (g) cudaGraphExecDestroy(g);
        if (st) cudaStreamSynchronize(st);
        cudaFree(ctrl);
        cudaFree(slots);
        cudaFree(args);
        cudaFree(offsets);
        cudaFree(seeds);
        if (ctrl_host) cudaFreeHost(ctrl_host);
        if (st) cudaStreamDestroy(st);
    }
};

template <class T> const void *batch_kernel_fn(bool hex)
{
    return hex ? (const void *)sweep_batch_kernel<T, true> : (const void *)sweep_batch_kernel<T, false>;
}

tf_status batch_setup(BatchRun &B, const tf_handle *problems, int32_t n)
{
    B.n = n;
    for (int k = 0; k < n; ++k) B.P.push_back(static_cast<Problem *>(reinterpret_cast<Object *>(problems[k])));
    B.device = B.P[0]->dev->device;
    B.fp64 = B.P[0]->dev->fp64;
    for (Problem *p : B.P) {
        if (p->dev->device != B.device || p->dev->fp64 != B.fp64)
            return fail(TF_ERR_ARG, "batched problems must share one device and one precision");
        if (p->opt.inject_stall) return fail(TF_ERR_ARG, "inject_stall is not supported in batched launches");
        if (p->reduce) return fail(TF_ERR_ARG, "a problem with a reduce function (direction sharding) cannot be batched");
        if (p->dev->n_lag > 0) return fail(TF_ERR_ARG, "a problem with lagged back edges cannot be batched");
        if (p->dev->schedule != TF_SCHED_AMT || p->dev->order != 1)
            return fail(TF_ERR_ARG, "batched launches run only linear tetrahedra and trilinear hexahedra with the "
                                    "TF_SCHED_AMT schedule");
        B.max_chunks = std::max(B.max_chunks, p->dev->n_chunks);
        B.warp_smem = std::max(B.warp_smem, p->dev->warp_smem);
    }
    TF_CUDA(cudaSetDevice(B.device));
    TF_CUDA(cudaDeviceGetAttribute(&B.sm_count, cudaDevAttrMultiProcessorCount, B.device));
    for (int c = 0; c < B.max_chunks; ++c) {
        size_t t = 0, s = 0;
        for (Problem *p : B.P) {
            DeviceState &d = *p->dev;
            if (c >= d.n_chunks) continue;
            t += (size_t)(d.chunk_task_begin[c + 1] - d.chunk_task_begin[c]);
            s += (size_t)(d.chunk_seed_begin[c + 1] - d.chunk_seed_begin[c]);
        }
        B.task_cap = std::max(B.task_cap, t);
        B.seed_cap = std::max(B.seed_cap, s);
    }
    if (B.task_cap >= (size_t(1) << 32)) return fail(TF_ERR_ARG, "batched launch of more than 2^32 tasks");
    const size_t argsz = B.fp64 ? sizeof(SweepArgs<double>) : sizeof(SweepArgs<float>);
    TF_CUDA(cudaMalloc(&B.ctrl, sizeof(Ctrl)));
    TF_CUDA(cudaMemset(B.ctrl, 0, sizeof(Ctrl)));
    TF_CUDA(cudaMallocHost(&B.ctrl_host, sizeof(Ctrl)));
    TF_CUDA(cudaMalloc(&B.slots, std::max<size_t>(B.task_cap, 1) * 8));
    TF_CUDA(cudaMemset(B.slots, 0, std::max<size_t>(B.task_cap, 1) * 8));
    TF_CUDA(cudaMalloc(&B.args, argsz * B.max_chunks * n));
    TF_CUDA(cudaMalloc(&B.offsets, 4 * (size_t)B.max_chunks * (n + 1)));
    TF_CUDA(cudaMalloc(&B.seeds, 4 * std::max<size_t>(B.seed_cap, 1) * B.max_chunks));
    TF_CUDA(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
    while (B.wpc > 1 && (size_t)B.warp_smem * B.wpc > 227 * 1024) B.wpc /= 2;
    const int dyn = (int)(B.warp_smem * B.wpc);
    for (Problem *p : B.P) B.hex = B.hex || p->dev->hex;
    const void *kfn = B.fp64 ? batch_kernel_fn<double>(B.hex) : batch_kernel_fn<float>(B.hex);
    TF_CUDA(ensure_dyn_smem(kfn, dyn));
    int per_sm = 0;
    TF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * B.wpc, dyn));
    B.grid = std::max(1, per_sm) * B.sm_count;
    return TF_OK;
}

// Per-chunk participant lists, global offsets, arguments and seeds of the active set.
template <class T> tf_status batch_build(BatchRun &B, const std::vector<char> &active)
{
    B.part.assign(B.max_chunks, {});
    B.n_tasks.assign(B.max_chunks, 0);
    B.n_seeds.assign(B.max_chunks, 0);
    std::vector<SweepArgs<T>> args((size_t)B.max_chunks * B.n);
    std::vector<uint32_t> offs((size_t)B.max_chunks * (B.n + 1), 0), seeds(std::max<size_t>(B.seed_cap, 1) * B.max_chunks);
    for (int c = 0; c < B.max_chunks; ++c) {
        uint32_t off = 0;
        size_t ns = 0;
        for (int k = 0; k < B.n; ++k) {
            Problem &p = *B.P[k];
            DeviceState &d = *p.dev;
            if (!active[k] || c >= d.n_chunks) continue;
            const int j = (int)B.part[c].size();
            B.part[c].push_back(k);
            SweepArgs<T> A = make_args<T>(p, c);
            A.ctrl = B.ctrl;  // waits report their errors to the batch's control block
            A.slots = B.slots;
            args[(size_t)c * B.n + j] = A;
            offs[(size_t)c * (B.n + 1) + j] = off;
            const int64_t s0 = d.chunk_seed_begin[c], s1 = d.chunk_seed_begin[c + 1];
            for (int64_t i = s0; i < s1; ++i)
                seeds[(size_t)c * B.seed_cap + ns++] = d.seeds_host[i] - (uint32_t)d.chunk_task_begin[c] + off;
            off += (uint32_t)(d.chunk_task_begin[c + 1] - d.chunk_task_begin[c]);
        }
        offs[(size_t)c * (B.n + 1) + B.part[c].size()] = off;
        B.n_tasks[c] = off;
        B.n_seeds[c] = ns;
    }
    TF_CUDA(cudaMemcpy(B.args, args.data(), sizeof(SweepArgs<T>) * args.size(), cudaMemcpyHostToDevice));
    TF_CUDA(cudaMemcpy(B.offsets, offs.data(), 4 * offs.size(), cudaMemcpyHostToDevice));
    TF_CUDA(cudaMemcpy(B.seeds, seeds.data(), 4 * seeds.size(), cudaMemcpyHostToDevice));
    return TF_OK;
}

// One source iteration of every active problem: phi_buf[k] -> phi_buf[1 - k].
template <class T>
tf_status batch_enqueue(BatchRun &B, const std::vector<char> &active, int k, bool with_stats, cudaStream_t st)
{
    for (int i = 0; i < B.n; ++i)
        if (active[i]) launch_source<T>(*B.P[i], B.P[i]->dev->phi_buf[k], st);
    for (int c = 0; c < B.max_chunks; ++c) {
        if (B.part[c].empty()) continue;
        begin_kernel<<<1, 1, 0, st>>>(B.ctrl, (unsigned long long)B.n_seeds[c], c == 0, 0);
        for (int i : B.part[c]) {
            DeviceState &d = *B.P[i]->dev;
            const int64_t t0 = d.chunk_task_begin[c], t1 = d.chunk_task_begin[c + 1];
            const int gb = d.chunk_group_begin[c], ng = d.chunk_group_begin[c + 1] - gb;
            const int fb = (int)std::min<int64_t>(std::max<int64_t>(1, (t1 - t0 + 255) / 256), (int64_t)d.sm_count * 8);
            fill_kernel<<<fb, 256, 0, st>>>(d.ctrl, d.counters, d.indeg, (uint32_t)t0, (uint32_t)(t1 - t0), d.slots,
                                            d.seeds, 0u, 0, d.group_rem + gb, d.group_total + gb, ng);
        }
        const int sb = (int)std::min<uint64_t>(std::max<uint64_t>(1, (B.n_seeds[c] + 255) / 256), (uint64_t)B.sm_count * 4);
        batch_seed_kernel<<<sb, 256, 0, st>>>(B.ctrl, B.slots, B.seeds + (size_t)c * B.seed_cap, (uint32_t)B.n_seeds[c]);
        BatchArgs<T> BA;
        BA.probs = reinterpret_cast<const SweepArgs<T> *>(B.args) + (size_t)c * B.n;
        BA.offsets = B.offsets + (size_t)c * (B.n + 1);
        BA.n = (int32_t)B.part[c].size();
        BA.ctrl = B.ctrl;
        BA.slots = B.slots;
        BA.n_tasks = B.n_tasks[c];
        BA.wait_limit_ns = (unsigned long long)(B.P[0]->opt.wait_limit_s * 1e9);
        BA.warp_smem = B.warp_smem;
        if (B.hex)
            sweep_batch_kernel<T, true><<<B.grid, 32 * B.wpc, (size_t)B.warp_smem * B.wpc, st>>>(BA);
        else
            sweep_batch_kernel<T, false><<<B.grid, 32 * B.wpc, (size_t)B.warp_smem * B.wpc, st>>>(BA);
        TF_CUDA(cudaGetLastError());
        end_kernel<<<1, 1, 0, st>>>(B.ctrl);
        for (int i : B.part[c]) launch_phi<T>(*B.P[i], c, B.P[i]->dev->phi_buf[1 - k], st);
    }
    if (with_stats) {
        for (int i = 0; i < B.n; ++i) {
            if (!active[i]) continue;
            Problem &p = *B.P[i];
            DeviceState &d = *p.dev;
            double *cur = d.phi_buf[k], *nxt = d.phi_buf[1 - k];
            launch_stats(p, cur, nxt, st);
            TF_CUDA(cudaMemcpyAsync(d.ctrl_host, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        }
    }
    TF_CUDA(cudaGetLastError());
    TF_CUDA(cudaMemcpyAsync(B.ctrl_host, B.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    return TF_OK;
}

template <class T> tf_status batch_capture(BatchRun &B, const std::vector<char> &active)
{
    for (auto &g : B.gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (int k = 0; k < 2; ++k) {
        if (cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
        const tf_status s = batch_enqueue<T>(B, active, k, true, B.st);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(B.st, &g);
        if (s != TF_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            break;
        }
        const cudaError_t ei = cudaGraphInstantiate(&B.gexec[k], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) B.gexec[k] = nullptr;
    }
    if (!B.gexec[0] || !B.gexec[1]) {
        for (auto &g : B.gexec)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        cudaGetLastError();
    }
    return TF_OK;
}

tf_status batch_check(BatchRun &B, const std::vector<char> &active)
{
    const Ctrl &c = *B.ctrl_host;
    if (c.error) {
        const int err = c.error;
        cudaMemsetAsync(&B.ctrl->error, 0, sizeof(int), B.st);
        cudaStreamSynchronize(B.st);
        return fail((tf_status)err, "batched sweep: device error");
    }
    // task counts accumulate over the chunk launches of one iteration
    uint64_t expect = 0;
    for (int ch = 0; ch < B.max_chunks; ++ch) expect += B.n_tasks[ch];
    (void)active;
    if (c.tasks_done != expect)
        return fail(TF_ERR_DEVICE, "batched sweep: executed " + std::to_string(c.tasks_done) + " of " +
                                       std::to_string(expect) + " tasks");
    return TF_OK;
}

tf_status copy_in(Problem &p, const double *src, double *dst, cudaStream_t st)
{
    const size_t bytes = (size_t)p.dev->C * p.dev->G * p.dev->nb * 8;
    if (!src) {
        TF_CUDA(cudaMemsetAsync(dst, 0, bytes, st));
        return TF_OK;
    }
    TF_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_pointer(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return TF_OK;
}

tf_status copy_out(Problem &p, const double *src, double *dst, cudaStream_t st)
{
    const size_t bytes = (size_t)p.dev->C * p.dev->G * p.dev->nb * 8;
    TF_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_pointer(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return TF_OK;
}

}  // namespace

tf_status device_batch_iterate(const tf_handle *problems, int32_t n, double tol, int32_t max_iters, double *const *phi,
                               tf_iter_info *info, bool stats_only_sweep, const double *const *phi_in, void *stream)
{
    BatchRun B;
    tf_status s = batch_setup(B, problems, n);
    if (s != TF_OK) return s;
    cudaStream_t user = (cudaStream_t)stream;
    cudaEvent_t ev = nullptr;
    TF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    TF_CUDA(cudaEventRecord(ev, user));
    TF_CUDA(cudaStreamWaitEvent(B.st, ev, 0));
    for (int i = 0; i < n; ++i) {
        const double *src = stats_only_sweep ? phi_in[i] : phi[i];
        if ((s = copy_in(*B.P[i], src, B.P[i]->dev->phi_buf[0], B.st)) != TF_OK) return s;
    }
    std::vector<char> active(n, 1), built;
    std::vector<int> iters(n, 0), final_buf(n, 0);
    std::vector<double> res(n, INFINITY), secs(n, 0.0), bals(n, 0.0);
    std::vector<char> conv(n, 0);
    const bool timing = !stats_only_sweep;
    int k = 0;
    const auto t0 = std::chrono::steady_clock::now();
    const int iterations = stats_only_sweep ? 1 : max_iters;
    for (int it = 1; it <= iterations; ++it) {
        if (active != built) {
            s = B.fp64 ? batch_build<double>(B, active) : batch_build<float>(B, active);
            if (s != TF_OK) return s;
            if (timing) {
                s = B.fp64 ? batch_capture<double>(B, active) : batch_capture<float>(B, active);
                if (s != TF_OK) return s;
            }
            built = active;
        }
        if (timing && B.gexec[k]) {
            TF_CUDA(cudaGraphLaunch(B.gexec[k], B.st));
        } else {
            s = B.fp64 ? batch_enqueue<double>(B, active, k, !stats_only_sweep, B.st)
                       : batch_enqueue<float>(B, active, k, !stats_only_sweep, B.st);
            if (s != TF_OK) return s;
        }
        TF_CUDA(cudaStreamSynchronize(B.st));
        if ((s = batch_check(B, active)) != TF_OK) return s;
        const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        bool any = false;
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            iters[i] = it;
            final_buf[i] = 1 - k;
            if (!stats_only_sweep) {
                std::memcpy(&res[i], &B.P[i]->dev->ctrl_host->residual_bits, sizeof(double));
                std::memcpy(&bals[i], &B.P[i]->dev->ctrl_host->balance_bits, sizeof(double));
                if (info && info[i].residual_history) info[i].residual_history[it - 1] = res[i];
                if (res[i] < tol) {
                    conv[i] = 1;
                    active[i] = 0;
                    secs[i] = now;
                }
            }
            if (active[i]) any = true;
        }
        for (int i = 0; i < n; ++i)
            if (!conv[i]) secs[i] = now;
        k = 1 - k;
        if (!any) break;
    }
    for (int i = 0; i < n; ++i) {
        DeviceState &d = *B.P[i]->dev;
        double *dst = stats_only_sweep ? const_cast<double *>(phi[i]) : phi[i];
        if ((s = copy_out(*B.P[i], d.phi_buf[final_buf[i]], dst, B.st)) != TF_OK) return s;
        if (!stats_only_sweep)
            TF_CUDA(cudaMemcpyAsync(d.gstats_host, d.gstats, sizeof(double) * 4 * d.G, cudaMemcpyDeviceToHost, B.st));
        d.last_chunk = d.n_chunks - 1;
    }
    TF_CUDA(cudaEventRecord(ev, B.st));
    TF_CUDA(cudaStreamWaitEvent(user, ev, 0));
    TF_CUDA(cudaStreamSynchronize(B.st));
    cudaEventDestroy(ev);
    bool all = true;
    for (int i = 0; i < n; ++i) {
        all = all && (conv[i] || stats_only_sweep);
        if (!info || stats_only_sweep) continue;
        DeviceState &d = *B.P[i]->dev;
        info[i].iterations = iters[i];
        info[i].converged = conv[i];
        info[i].residual = res[i];
        info[i].balance = bals[i];
        info[i].seconds = secs[i];
        double tot = 0.0;
        for (int g = 0; g < d.G; ++g) {
            tot += d.gstats_host[4 * g + 1];
            if (info[i].integrated_flux) info[i].integrated_flux[g] = d.gstats_host[4 * g + 1];
        }
        info[i].integrated_total = tot;
    }
    return all ? TF_OK : fail(TF_ERR_NOT_CONVERGED, "batched source iteration reached max_iters");
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
    if (d.hex) {
        if (d.fp64)
            psi_ho_out_kernel<double, 8><<<blocks, 256, 0, st>>>((const double *)d.psi + (size_t)(dir - a0) * CG * 8,
                                                                 (double *)out, d.C, d.G);
        else
            psi_ho_out_kernel<float, 8><<<blocks, 256, 0, st>>>((const float *)d.psi + (size_t)(dir - a0) * CG * 8,
                                                                (float *)out, d.C, d.G);
    } else if (d.order == 3) {
        if (d.fp64)
            psi_ho_out_kernel<double, 20><<<blocks, 256, 0, st>>>((const double *)d.psi + (size_t)(dir - a0) * CG * 20,
                                                                  (double *)out, d.C, d.G);
        else
            psi_ho_out_kernel<float, 20><<<blocks, 256, 0, st>>>((const float *)d.psi + (size_t)(dir - a0) * CG * 20,
                                                                 (float *)out, d.C, d.G);
    } else if (d.order == 2) {
        if (d.fp64)
            psi_ho_out_kernel<double, 10><<<blocks, 256, 0, st>>>((const double *)d.psi + (size_t)(dir - a0) * CG * 10,
                                                                  (double *)out, d.C, d.G);
        else
            psi_ho_out_kernel<float, 10><<<blocks, 256, 0, st>>>((const float *)d.psi + (size_t)(dir - a0) * CG * 10,
                                                                 (float *)out, d.C, d.G);
    } else if (d.paired)
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
