// Per-iteration kernels of the higher-order elements (NB = 10 nodes: quadratic,
// NB = 20: cubic): source update, phi reduction, boundary leakage, FP64 statistics
// and stopping test, psi inspection.  Included by sweep.cu inside namespace tf,
// after the linear element's kernels (it uses WeightPair, two_sum_acc, BalIn,
// record_balance, kFourPi).
//
// Layouts: caller phi and Q [C][G][NB] (FP64); device Q, q [C][NB][G] and psi
// [Dc][C][NB][G] in the sweep precision (node-major, so that lanes over groups read
// and write whole lines).  Element tables (exact, per order): pw[i] = int phi_i / V;
// for the face opposite vertex f its NF nodes fn[f][.] and fav[.] = int_f phi / A
// (the same in every face's node order).
#pragma once

struct HoTables {
    const double *pw;      // [NB]
    const int32_t *fn;     // [4][NF]
    const double *fav;     // [NF]
};

// q[c][i][g] = (Q[c][i][g] + sum_h sigma_s[m][h][g] phi[c][h][i]) / 4 pi.  One CTA
// stages the scalar flux of a few cells (in the sweep precision) in shared memory.
template <class T, int NB>
__global__ void __launch_bounds__(256) source_ho_kernel(const double *__restrict__ phi, const T *__restrict__ Qext,
                                                        const T *__restrict__ sigma_s, const int32_t *__restrict__ mat,
                                                        T *__restrict__ q, int64_t C, int G, int cells_per_cta)
{
    extern __shared__ unsigned char smem_raw[];
    T *ph = reinterpret_cast<T *>(smem_raw);  // [cells_per_cta][G][NB]
    const T inv4pi = T(1.0 / (4.0 * 3.14159265358979323846));
    for (int64_t c0 = (int64_t)blockIdx.x * cells_per_cta; c0 < C; c0 += (int64_t)gridDim.x * cells_per_cta) {
        const int nc = (int)((C - c0) < (int64_t)cells_per_cta ? (C - c0) : (int64_t)cells_per_cta);
        __syncthreads();
        for (int e = threadIdx.x; e < nc * G * NB; e += blockDim.x) ph[e] = (T)phi[(size_t)c0 * G * NB + e];
        __syncthreads();
        for (int u = threadIdx.x; u < nc * G; u += blockDim.x) {
            const int lc = u / G, g = u - lc * G;
            const int64_t c = c0 + lc;
            const T *S = sigma_s + (size_t)__ldg(mat + c) * G * G + g;
            const T *p = ph + (size_t)lc * G * NB;
            T a[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) a[i] = T(0);
            for (int h = 0; h < G; ++h) {
                const T s = __ldg(S + (size_t)h * G);
#pragma unroll
                for (int i = 0; i < NB; ++i) a[i] += s * p[NB * h + i];
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const size_t at = ((size_t)c * NB + i) * G + g;
                q[at] = (__ldg(Qext + at) + a[i]) * inv4pi;
            }
        }
    }
}

// phi[c][g][i] (+)= sum over the chunk's directions of w_a psi_a[c][i][g] (Eq. (2)).
// Thread per (cell, group); FP32 psi with PAIR: exact float-pair products and sums
// (as the linear element's phi_kernel), rounded once to FP64.
template <class T, bool PAIR, int NB>
__global__ void __launch_bounds__(256) phi_ho_kernel(const T *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                     int Dc, int64_t C, int G, double *__restrict__ phi, int accumulate)
{
    const size_t CG = (size_t)C * G;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < CG; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx / (size_t)G;
        const int g = (int)(idx - c * (size_t)G);
        const T *src = psi + c * NB * (size_t)G + g;
        double r[NB];
        if constexpr (PAIR) {
            float hi[NB], lo[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) hi[i] = lo[i] = 0.f;
            for (int a = 0; a < Dc; ++a) {
                const T *s = src + (size_t)a * CG * NB;
                const WeightPair w = wts[a];
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const float x = __ldcs(s + (size_t)i * G);
                    const float pp = w.hi * x;
                    const float e = fmaf(w.hi, x, -pp) + w.lo * x;
                    two_sum_acc(hi[i], lo[i], pp, e);
                }
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) r[i] = (double)hi[i] + (double)lo[i];
        } else {
#pragma unroll
            for (int i = 0; i < NB; ++i) r[i] = 0.0;
            for (int a = 0; a < Dc; ++a) {
                const T *s = src + (size_t)a * CG * NB;
                const double w = wts[a].d;
#pragma unroll
                for (int i = 0; i < NB; ++i) r[i] = fma(w, (double)__ldcs(s + (size_t)i * G), r[i]);
            }
        }
        double *out = phi + idx * NB;
#pragma unroll
        for (int i = 0; i < NB; ++i) out[i] = accumulate ? out[i] + r[i] : r[i];
    }
}

// Boundary leakage (vacuum boundaries): per (boundary cell, group) over the chunk's
// directions, w_a s_f <psi_a>_f on every boundary outflow face (s_f = Omega_a . N_f
// not below the sweep graph's inflow threshold -1e-12 |N_f|), with the face average
// <psi>_f = sum_r fav[r] psi[fn[f][r]].  Accumulated as the linear element's leak_kernel.
template <class T, int NB, int NF, class Geo>
__global__ void __launch_bounds__(256) leak_ho_kernel(const T *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                      const V4<T> *__restrict__ omega, int Dc, int64_t C, int G,
                                                      const uint32_t *__restrict__ bcells, int64_t nb,
                                                      const Geo *__restrict__ geo, HoTables tb, double *__restrict__ leak)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nb * G; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = u / G;
        const int g = (int)(u - b * G);
        const uint32_t c = bcells[b];
        const Geo &cg = geo[c];
        uint32_t faces = 0;
        T nx[4], ny[4], nz[4], thr[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            faces |= (cg.nbr[f] < 0 ? 1u : 0u) << f;
            nx[f] = cg.nrm[3 * f];
            ny[f] = cg.nrm[3 * f + 1];
            nz[f] = cg.nrm[3 * f + 2];
            thr[f] = T(-1e-12) * sqrt(nx[f] * nx[f] + ny[f] * ny[f] + nz[f] * nz[f]);
        }
        double acc = 0.0;
        float hi = 0.f, lo = 0.f;
        for (int a = 0; a < Dc; ++a) {
            const T *s = psi + (((size_t)a * C + c) * NB) * G + g;
            const V4<T> om = omega[a];
            T t = T(0);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (!((faces >> f) & 1u)) continue;
                const T sf = om.x * nx[f] + om.y * ny[f] + om.z * nz[f];
                if (sf < thr[f]) continue;  // inflow face of a vacuum boundary
                T avg = T(0);
                for (int r = 0; r < NF; ++r)
                    avg += T(__ldg(tb.fav + r)) * s[(size_t)__ldg(tb.fn + NF * f + r) * G];
                t += sf * avg;
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

// Boundary leakage of trilinear hexahedra: per (boundary cell, group) over the chunk's
// directions, w_a sum over the boundary faces f of int_f (Omega_a . N) psi =
// sum_k psi_k sum_d Omega_d sum_l F[f][d][l][k], psi the cell's own nodal values on an
// outflow face (Omega_a . Nbar_f not below the sweep graph's inflow threshold
// -1e-12 |Nbar_f|) and the prescribed inflow at the face's vertices on an inflow face
// (vacuum, psi_in NULL: nothing).
template <class T>
__global__ void __launch_bounds__(256) leak_hex_kernel(const T *__restrict__ psi, const WeightPair *__restrict__ wts,
                                                       const V4<T> *__restrict__ omega, int Dc, int64_t C, int G,
                                                       const uint32_t *__restrict__ bcells, int64_t nb,
                                                       const HexGeo<T> *__restrict__ geo, const int32_t *__restrict__ hexv,
                                                       const T *__restrict__ psi_in, double *__restrict__ leak)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nb * G; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = u / G;
        const int g = (int)(u - b * G);
        const uint32_t c = bcells[b];
        const HexGeo<T> &cg = geo[c];
        double acc = 0.0;
        float hi = 0.f, lo = 0.f;
        for (int a = 0; a < Dc; ++a) {
            const T *s = psi + (((size_t)a * C + c) * 8) * G + g;
            const V4<T> om = omega[a];
            T t = T(0);
            for (int f = 0; f < 6; ++f) {
                if (cg.nbr[f] >= 0) continue;
                const T nx = cg.nbar[f][0], ny = cg.nbar[f][1], nz = cg.nbar[f][2];
                const T sf = om.x * nx + om.y * ny + om.z * nz;
                const bool in = sf < T(-1e-12) * sqrt(nx * nx + ny * ny + nz * nz);
                if (in && !psi_in) continue;  // inflow face of a vacuum boundary
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    T col = T(0);
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        col += om.x * cg.F[f][0][4 * l + k] + om.y * cg.F[f][1][4 * l + k] + om.z * cg.F[f][2][4 * l + k];
                    const int v = hex_node(f, k);
                    t += col * (in ? psi_in[(size_t)hexv[8 * (size_t)c + v] * G + g] : s[(size_t)v * G]);
                }
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

// The statistics of stats_kernel / stats_res_kernel for a higher-order field (same
// partial layout, so the same finish kernels apply): integral sum_c V_c sum_i pw_i phi_i
// (Eq. (3)), plain nodal sum, absorption, source, max |phi| and (RES) max |dphi|.  With
// per-cell weights pwc [C][NB] (hexahedra: int b_i), the integral is sum_c sum_i pwc phi_i.
template <class T, bool RES, int NB>
__global__ void __launch_bounds__(256) stats_ho_kernel(const double *__restrict__ phi_new,
                                                       const double *__restrict__ phi_old,
                                                       const double *__restrict__ vol, int64_t C, int G,
                                                       double *__restrict__ part, BalIn bi, const double *__restrict__ pw,
                                                       const double *__restrict__ pwc)
{
    constexpr int NP = RES ? 6 : 5;
    __shared__ double sh[NP][8][32];
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + threadIdx.x;
        double mx = 0.0, iv = 0.0, pl = 0.0, dm = 0.0, ab = 0.0, sr = 0.0;
        if (g < G) {
            for (int64_t c = (int64_t)blockIdx.x * 8 + threadIdx.y; c < C; c += (int64_t)gridDim.x * 8) {
                const double *pn = phi_new + ((size_t)c * G + g) * NB;
                double plain = 0.0, ws = 0.0, qs = 0.0;
                const T *q = reinterpret_cast<const T *>(bi.q) + (size_t)c * NB * G + g;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const double w = pwc ? __ldg(pwc + (size_t)c * NB + i) : __ldg(pw + i);
                    mx = fmax(mx, fabs(pn[i]));
                    plain += pn[i];
                    ws += w * pn[i];
                    qs += w * (double)q[(size_t)i * G];
                }
                if constexpr (RES) {
                    const double *po = phi_old + ((size_t)c * G + g) * NB;
#pragma unroll
                    for (int i = 0; i < NB; ++i) dm = fmax(dm, fabs(pn[i] - po[i]));
                }
                const double vc = pwc ? 1.0 : vol[c];
                iv += vc * ws;
                pl += plain;
                ab += bi.sig[(size_t)bi.mat[c] * G + g] * vc * ws;
                sr += vc * kFourPi * qs;
            }
        }
        const double vals[6] = {mx, iv, pl, RES ? dm : ab, RES ? ab : sr, sr};
#pragma unroll
        for (int k = 0; k < NP; ++k) sh[k][threadIdx.y][threadIdx.x] = vals[k];
        __syncthreads();
        if (threadIdx.y == 0 && g < G) {
            double o[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) o[k] = sh[k][0][threadIdx.x];
            for (int y = 1; y < 8; ++y) {
                o[0] = fmax(o[0], sh[0][y][threadIdx.x]);
                o[1] += sh[1][y][threadIdx.x];
                o[2] += sh[2][y][threadIdx.x];
                if constexpr (RES) {
                    o[3] = fmax(o[3], sh[3][y][threadIdx.x]);
                    o[4] += sh[4][y][threadIdx.x];
                    o[5] += sh[5][y][threadIdx.x];
                } else {
                    o[3] += sh[3][y][threadIdx.x];
                    o[4] += sh[4][y][threadIdx.x];
                }
            }
            double *dst = part + ((size_t)blockIdx.x * G + g) * NP;
#pragma unroll
            for (int k = 0; k < NP; ++k) dst[k] = o[k];
        }
        __syncthreads();
    }
}

// Pointwise stopping test (residual_floor < 1) for a higher-order field, as residual_kernel.
template <int NB>
__global__ void __launch_bounds__(256) residual_ho_kernel(const double *__restrict__ phi_new,
                                                          const double *__restrict__ phi_old,
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
            const double *pn = phi_new + ((size_t)c * G + g) * NB, *po = phi_old + ((size_t)c * G + g) * NB;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const double diff = fabs(pn[i] - po[i]);
                if (diff == 0.0) continue;
                const double den = fmax(fabs(pn[i]), floor_);
                rmax = fmaxf(rmax, den > 0.0 ? __fdiv_rn((float)(diff * inv), (float)(den * inv)) : INFINITY);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if ((threadIdx.x & 31) == 0 && rmax > 0.f)
        atomicMax(&ctrl->residual_bits, (unsigned long long)__double_as_longlong((double)rmax));
}

// psi of one direction, [C][NB][G] -> the caller's [C][G][NB] (inspection only).
template <class T, int NB>
__global__ void psi_ho_out_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t C, int G)
{
    const size_t n = (size_t)C * G * NB;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t c = idx / ((size_t)G * NB);
        const size_t r = idx - c * (size_t)G * NB;
        const int g = (int)(r / NB), i = (int)(r - (size_t)g * NB);
        dst[idx] = src[(c * NB + i) * G + g];
    }
}
