// Learned initial flux: a per-cell multilayer perceptron that proposes the
// starting scalar flux of source iteration (the paper's iteration starts from
// a given flux; this network only chooses it, the stopping test decides the
// answer).  Inputs -> H -> H -> outputs with tanh hidden activations; weights
// stored in BF16 for the forward and backward passes, FP32 master copy for
// Adam, FP32 accumulation throughout.  Every step (features, targets,
// forward, backward, weight gradients, Adam, prediction) is a kernel here.
//
// Master parameters, flat FP32: W1 [H][I], b1 [H], W2 [H][H], b2 [H],
// W3 [O][H], b3 [O].  The BF16 copy used by the kernels holds W1^T [I][H],
// W2^T [H][H] and W3 [O][H] (the orders the per-sample loops read).
// Loss over n samples: (1/(n O)) sum_s sum_o w_so (y_so - (t_so - mu)/sd)^2, with
// (mu, sd) the target standardisation kept in the handle and w optional
// per-target weights (1 without them) times kappa on overshooting outputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/tflearn.h"
#include "tf_internal.h"

namespace tf {

namespace {

constexpr int kKC = 32;          // W1^T rows staged per chunk of the forward pass
constexpr int kMaxO = 64;        // outputs
constexpr int kMaxSplits = 64;   // sample splits of the weight-gradient reduction
constexpr int kGT = 64;          // weight-gradient tile (rows and columns)
constexpr int kGK = 16;          // samples per staged slice of that tile

}  // namespace

struct Mlp : Object {
    Mlp() : Object(Kind::Mlp) {}
    ~Mlp() override;
    int I = 0, H = 0, O = 0;
    size_t np = 0;
    int device = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // master params, Adam moments, gradient
    __nv_bfloat16 *wb = nullptr;
    float *act = nullptr;      // per-sample scratch: A1, A2, D1, D2 [n][H], Y, DY [n][O]
    size_t act_cap = 0;
    float *part = nullptr;     // weight-gradient partial sums [splits][R][C+1]
    float *loss = nullptr;     // [0] last minibatch loss, [1] epoch accumulator
    double *red = nullptr;     // reduction scratch (2 doubles)
    float *xm = nullptr, *xinv = nullptr;  // input standardisation x' = (x - xm) xinv, [I] (NULL: none)
    float *xn = nullptr;       // standardised inputs of a gradient call [n][I]
    size_t xn_cap = 0;
    float mu = 0.f, sd = 1.f;
    float kappa = 1.f;             // loss weight multiplier of overshooting outputs
    float t_cap = INFINITY;        // predictions are capped at this target value
    float shrink = 1.f;            // the predicted flux is multiplied by this factor
    int64_t step = 0;
    size_t off_b1() const { return (size_t)H * I; }
    size_t off_W2() const { return off_b1() + H; }
    size_t off_b2() const { return off_W2() + (size_t)H * H; }
    size_t off_W3() const { return off_b2() + H; }
    size_t off_b3() const { return off_W3() + (size_t)O * H; }
};

Mlp::~Mlp()
{
    cudaSetDevice(device);
    cudaFree(p);
    cudaFree(m);
    cudaFree(v);
    cudaFree(g);
    cudaFree(wb);
    cudaFree(act);
    cudaFree(part);
    cudaFree(loss);
    cudaFree(red);
    cudaFree(xm);
    cudaFree(xinv);
    cudaFree(xn);
}

namespace {

#define MLP_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? TF_ERR_NOMEM : TF_ERR_CUDA,                   \
                        std::string("mlp.cu:") + std::to_string(__LINE__) + " " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------- features
// Per cell, I = G^2 + 4G values:
//   [0, G)            log sigma_t[m][g]
//   [G, G + G^2)      sigma_s[m][g'][g] / sigma_t[m][g'] at G + g' G + g (scattering probabilities)
//   next G            log(qbar[g] + 1e-6), qbar = cell-average source = mean of the 4 nodal Q[c][g][i]
//   next G            mean over the face neighbours of log sigma_t[g] (the cell's own value if none)
//   next G            log(mean over the face neighbours of qbar[g] + 1e-6) (the cell's own qbar if none)
// (the flux grows linearly with the source, so its logarithm, the target, with log qbar)
__global__ void features_kernel(int64_t C, int G, const int32_t *__restrict__ mat, const double *__restrict__ sig_t,
                                const double *__restrict__ sig_s, const double *__restrict__ Q,
                                const int32_t *__restrict__ nbr, float *__restrict__ X, int ld)
{
    const int I = G * G + 4 * G;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; c < C; c += (int64_t)gridDim.x * blockDim.y) {
        const int m = mat[c];
        float *x = X + (size_t)c * ld;
        int nb[4], nn = 0;
        for (int f = 0; f < 4; ++f) {
            const int n = nbr[4 * c + f];
            if (n >= 0) nb[nn++] = n;
        }
        for (int e = threadIdx.x; e < I; e += blockDim.x) {
            double val;
            if (e < G) {
                val = log(sig_t[(size_t)m * G + e]);
            } else if (e < G + G * G) {
                const int k = e - G, gf = k / G, gt = k - gf * G;
                val = sig_s[((size_t)m * G + gf) * G + gt] / sig_t[(size_t)m * G + gf];
            } else if (e < 2 * G + G * G) {
                const double *q = Q + ((size_t)c * G + (e - G - G * G)) * 4;
                val = log(0.25 * (((q[0] + q[1]) + q[2]) + q[3]) + 1e-6);
            } else if (e < 3 * G + G * G) {
                const int gg = e - 2 * G - G * G;
                double s = 0.0;
                for (int k = 0; k < nn; ++k) s += log(sig_t[(size_t)mat[nb[k]] * G + gg]);
                val = nn ? s / nn : log(sig_t[(size_t)m * G + gg]);
            } else {
                const int gg = e - 3 * G - G * G;
                double s = 0.0;
                for (int k = 0; k < nn; ++k) {
                    const double *q = Q + ((size_t)nb[k] * G + gg) * 4;
                    s += 0.25 * (((q[0] + q[1]) + q[2]) + q[3]);
                }
                const double *q = Q + ((size_t)c * G + gg) * 4;
                val = log((nn ? s / nn : 0.25 * (((q[0] + q[1]) + q[2]) + q[3])) + 1e-6);
            }
            x[e] = (float)val;
        }
    }
}

// Context inputs: fields per (cell, group) averaged over wider neighbourhoods.  One round of
// neighbour averaging replaces a cell's value by the mean of its own and its face neighbours'
// values (a diffusion step on the cell graph: after t rounds a value has spread over about
// sqrt(t) cells).
__global__ void smooth_kernel(int64_t C, int G, const int32_t *__restrict__ nbr, const double *__restrict__ in,
                              double *__restrict__ out)
{
    const int64_t CG = C * G;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < CG; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / G;
        const int g = (int)(i - c * G);
        double s = in[i];
        int n = 1;
        for (int f = 0; f < 4; ++f) {
            const int32_t nb = nbr[4 * c + f];
            if (nb >= 0) {
                s += in[(size_t)nb * G + g];
                ++n;
            }
        }
        out[i] = s / n;
    }
}

// The starting fields of the context: cell-average source qbar and log sigma_t per (cell, group).
__global__ void context_init_kernel(int64_t C, int G, const int32_t *__restrict__ mat, const double *__restrict__ sig_t,
                                    const double *__restrict__ Q, double *__restrict__ vq, double *__restrict__ vs)
{
    const int64_t CG = C * G;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < CG; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / G;
        const int g = (int)(i - c * G);
        const double *q = Q + (size_t)i * 4;
        vq[i] = 0.25 * (((q[0] + q[1]) + q[2]) + q[3]);
        vs[i] = log(sig_t[(size_t)mat[c] * G + g]);
    }
}

// Columns [col, col + G) of X: log(vq + 1e-6); [col + G, col + 2G): vs.
__global__ void context_write_kernel(int64_t C, int G, int ld, int col, const double *__restrict__ vq,
                                     const double *__restrict__ vs, float *__restrict__ X)
{
    const int64_t CG = C * G;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < CG; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / G;
        const int g = (int)(i - c * G);
        X[(size_t)c * ld + col + g] = (float)log(vq[i] + 1e-6);
        X[(size_t)c * ld + col + G + g] = (float)vs[i];
    }
}

// Training target per (cell, group): log(max(cell-average phi, 0) + 1e-6); the
// cell average of a linear function on a tetrahedron is the mean of its 4 nodal values.
__global__ void targets_kernel(int64_t CG, const double *__restrict__ phi, float *__restrict__ T)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < CG; e += (int64_t)gridDim.x * blockDim.x) {
        const double *f = phi + (size_t)e * 4;
        const double avg = 0.25 * (((f[0] + f[1]) + f[2]) + f[3]);
        T[e] = (float)log(fmax(avg, 0.0) + 1e-6);
    }
}

// Per-group maximum of the clamped cell-average flux (FP64 bit patterns of non-negative
// values order like the values, so an unsigned atomicMax finds the maximum).
__global__ void group_max_kernel(int64_t C, int G, const double *__restrict__ phi, unsigned long long *__restrict__ gmax)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C * G; e += (int64_t)gridDim.x * blockDim.x) {
        const double *f = phi + (size_t)e * 4;
        const double avg = fmax(0.25 * (((f[0] + f[1]) + f[2]) + f[3]), 0.0);
        atomicMax(gmax + (e % G), (unsigned long long)__double_as_longlong(avg));
    }
}

// w[c][g] = (phi_cg / max_c phi_cg)^2 + floor, phi the clamped cell average (floor alone
// where the group's maximum is 0).
__global__ void weights_kernel(int64_t C, int G, const double *__restrict__ phi,
                               const unsigned long long *__restrict__ gmax, float floor_w, float *__restrict__ W)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C * G; e += (int64_t)gridDim.x * blockDim.x) {
        const double *f = phi + (size_t)e * 4;
        const double avg = fmax(0.25 * (((f[0] + f[1]) + f[2]) + f[3]), 0.0);
        const double m = __longlong_as_double((long long)gmax[e % G]);
        const double r = m > 0.0 ? avg / m : 0.0;
        W[e] = (float)(r * r + (double)floor_w);
    }
}

// sum of (t - shift)^2 (square = 1) or of t - shift (square = 0) over n values into acc (FP64)
__global__ void moment_kernel(int64_t n, const float *__restrict__ T, double shift, int square, double *__restrict__ acc)
{
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)T[e] - shift;
        s += square ? d * d : d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// Per column k of X [n][I]: acc[k] += sum over rows of (x - shift[k]) (square = 0) or its
// square (square = 1); FP64.  Threads span the columns of a row (coalesced), blocks stride rows.
__global__ void colsum_kernel(int64_t n, int I, const float *__restrict__ X, const double *__restrict__ shift,
                              int square, double *__restrict__ acc)
{
    for (int k = threadIdx.x; k < I; k += blockDim.x) {
        const double sh = shift ? shift[k] : 0.0;
        double s = 0.0;
        for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
            const double d = (double)X[(size_t)r * I + k] - sh;
            s += square ? d * d : d;
        }
        atomicAdd(acc + k, s);
    }
}

// mean[k] = sum[k] / n; then, from the squared deviations, inv[k] = 1 / std (1 for a constant column).
__global__ void colstat_kernel(int I, int64_t n, const double *__restrict__ sum, const double *__restrict__ sq,
                               double *__restrict__ mean_d, float *__restrict__ mean, float *__restrict__ inv, int stage)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I; k += gridDim.x * blockDim.x) {
        if (stage == 0) {
            mean_d[k] = sum[k] / (double)n;
            mean[k] = (float)mean_d[k];
        } else {
            const double var = sq[k] / (double)n;
            inv[k] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.f;
        }
    }
}

// Xn[s][k] = (X[s][k] - xm[k]) xinv[k].
__global__ void normalize_kernel(int64_t n, int I, const float *__restrict__ X, const float *__restrict__ xm,
                                 const float *__restrict__ xinv, float *__restrict__ Xn)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * I; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % I);
        Xn[e] = (X[e] - xm[k]) * xinv[k];
    }
}

// Largest of n values into *acc as an order-preserving unsigned key of the float.
__device__ __forceinline__ unsigned float_key(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__global__ void max_key_kernel(int64_t n, const float *__restrict__ T, unsigned *__restrict__ acc)
{
    unsigned k = 0u;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        k = max(k, float_key(T[e]));
    for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
    if ((threadIdx.x & 31) == 0) atomicMax(acc, k);
}

// ---------------------------------------------------------------- forward
// One thread per sample; the BF16 weights are widened to FP32 in shared memory
// (W1^T in chunks of kKC rows) and read as float4 broadcasts.  With xm / xinv the
// inputs are standardised on load.
template <int H>
__global__ void __launch_bounds__(128) forward_kernel(int64_t n, int I, int O, const __nv_bfloat16 *__restrict__ wb,
                                                      const float *__restrict__ P, const float *__restrict__ X,
                                                      const float *__restrict__ xm, const float *__restrict__ xinv,
                                                      float *__restrict__ Y, float *__restrict__ A1,
                                                      float *__restrict__ A2)
{
    extern __shared__ __align__(16) float fsm[];
    float *w1c = fsm, *w2t = w1c + kKC * H, *w3 = w2t + H * H, *bb = w3 + O * H;
    const __nv_bfloat16 *W1T = wb, *W2T = wb + (size_t)I * H, *W3 = W2T + H * H;
    const float *b1 = P + (size_t)H * I, *b2 = b1 + H + H * H, *b3 = b2 + H + (size_t)O * H;
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) w2t[k] = __bfloat162float(W2T[k]);
    for (int k = threadIdx.x; k < O * H; k += blockDim.x) w3[k] = __bfloat162float(W3[k]);
    for (int k = threadIdx.x; k < 2 * H + O; k += blockDim.x) bb[k] = k < H ? b1[k] : (k < 2 * H ? b2[k - H] : b3[k - 2 * H]);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < n;
    const float *x = X + (size_t)(live ? s : 0) * I;
    __syncthreads();
    float h[H];
#pragma unroll
    for (int j = 0; j < H; ++j) h[j] = bb[j];
    for (int k0 = 0; k0 < I; k0 += kKC) {
        const int kn = min(kKC, I - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * H; e += blockDim.x) w1c[e] = __bfloat162float(W1T[(size_t)k0 * H + e]);
        __syncthreads();
        if (live)
            for (int kk = 0; kk < kn; ++kk) {
                const float xk = xm ? (x[k0 + kk] - __ldg(xm + k0 + kk)) * __ldg(xinv + k0 + kk) : x[k0 + kk];
                const float4 *wr = reinterpret_cast<const float4 *>(w1c + kk * H);
#pragma unroll
                for (int q = 0; q < H / 4; ++q) {
                    const float4 w = wr[q];
                    h[4 * q + 0] = fmaf(w.x, xk, h[4 * q + 0]);
                    h[4 * q + 1] = fmaf(w.y, xk, h[4 * q + 1]);
                    h[4 * q + 2] = fmaf(w.z, xk, h[4 * q + 2]);
                    h[4 * q + 3] = fmaf(w.w, xk, h[4 * q + 3]);
                }
            }
    }
    if (!live) return;
#pragma unroll
    for (int j = 0; j < H; ++j) h[j] = tanhf(h[j]);
    if (A1) {
        float4 *a = reinterpret_cast<float4 *>(A1 + (size_t)s * H);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) a[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
    }
    float h2[H];
#pragma unroll
    for (int j = 0; j < H; ++j) h2[j] = bb[H + j];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const float4 *wr = reinterpret_cast<const float4 *>(w2t + k * H);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            const float4 w = wr[q];
            h2[4 * q + 0] = fmaf(w.x, h[k], h2[4 * q + 0]);
            h2[4 * q + 1] = fmaf(w.y, h[k], h2[4 * q + 1]);
            h2[4 * q + 2] = fmaf(w.z, h[k], h2[4 * q + 2]);
            h2[4 * q + 3] = fmaf(w.w, h[k], h2[4 * q + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < H; ++j) h2[j] = tanhf(h2[j]);
    if (A2) {
        float4 *a = reinterpret_cast<float4 *>(A2 + (size_t)s * H);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) a[q] = make_float4(h2[4 * q], h2[4 * q + 1], h2[4 * q + 2], h2[4 * q + 3]);
    }
    for (int o = 0; o < O; ++o) {
        const float4 *wr = reinterpret_cast<const float4 *>(w3 + o * H);
        float acc = bb[2 * H + o];
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            const float4 w = wr[q];
            acc = fmaf(w.x, h2[4 * q + 0], acc);
            acc = fmaf(w.y, h2[4 * q + 1], acc);
            acc = fmaf(w.z, h2[4 * q + 2], acc);
            acc = fmaf(w.w, h2[4 * q + 3], acc);
        }
        Y[(size_t)s * O + o] = acc;
    }
}

// ---------------------------------------------------------------- backward
// Per sample, r_o = y_o - (t_o - mu)/sd: dy_o = 2 w_o r_o / (n O), with w_o the given weight
// (1 without weights) times kappa where r_o > 0 (an overshooting output);
// d2 = (W3^T dy) (1 - a2^2); d1 = (W2^T d2) (1 - a1^2), with the BF16 weights of the forward pass.
// loss[0] += minibatch loss; loss[1] += weighted squared error / (n_epoch O) when n_epoch > 0.
template <int H>
__global__ void __launch_bounds__(128) backward_kernel(int64_t n, int I, int O, const __nv_bfloat16 *__restrict__ wb,
                                                       const float *__restrict__ Y, const float *__restrict__ T,
                                                       const float *__restrict__ Wt, float mu, float inv_sd, float kappa,
                                                       const float *__restrict__ A1,
                                                       const float *__restrict__ A2, float *__restrict__ DY,
                                                       float *__restrict__ D1, float *__restrict__ D2,
                                                       float *__restrict__ loss, int64_t n_epoch)
{
    extern __shared__ __align__(16) float fsm[];
    float *w2t = fsm, *w3 = w2t + H * H;
    const __nv_bfloat16 *W2T = wb + (size_t)I * H, *W3 = W2T + H * H;
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) w2t[k] = __bfloat162float(W2T[k]);
    for (int k = threadIdx.x; k < O * H; k += blockDim.x) w3[k] = __bfloat162float(W3[k]);
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float scale = 2.f / ((float)n * (float)O);
    float lsum = 0.f;
    if (s < n) {
        float d2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) d2[k] = 0.f;
        for (int o = 0; o < O; ++o) {
            const float r = Y[(size_t)s * O + o] - (T[(size_t)s * O + o] - mu) * inv_sd;
            const float w = (Wt ? Wt[(size_t)s * O + o] : 1.f) * (r > 0.f ? kappa : 1.f);
            lsum = fmaf(w * r, r, lsum);
            const float dy = scale * w * r;
            DY[(size_t)s * O + o] = dy;
            const float4 *wr = reinterpret_cast<const float4 *>(w3 + o * H);
#pragma unroll
            for (int q = 0; q < H / 4; ++q) {
                const float4 w = wr[q];
                d2[4 * q + 0] = fmaf(w.x, dy, d2[4 * q + 0]);
                d2[4 * q + 1] = fmaf(w.y, dy, d2[4 * q + 1]);
                d2[4 * q + 2] = fmaf(w.z, dy, d2[4 * q + 2]);
                d2[4 * q + 3] = fmaf(w.w, dy, d2[4 * q + 3]);
            }
        }
        const float4 *a2 = reinterpret_cast<const float4 *>(A2 + (size_t)s * H);
        float4 *o2 = reinterpret_cast<float4 *>(D2 + (size_t)s * H);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            const float4 z = a2[q];
            d2[4 * q + 0] *= 1.f - z.x * z.x;
            d2[4 * q + 1] *= 1.f - z.y * z.y;
            d2[4 * q + 2] *= 1.f - z.z * z.z;
            d2[4 * q + 3] *= 1.f - z.w * z.w;
            o2[q] = make_float4(d2[4 * q], d2[4 * q + 1], d2[4 * q + 2], d2[4 * q + 3]);
        }
        const float *a1 = A1 + (size_t)s * H;
        float *o1 = D1 + (size_t)s * H;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float4 *wr = reinterpret_cast<const float4 *>(w2t + k * H);
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < H / 4; ++q) {
                const float4 w = wr[q];
                acc = fmaf(w.x, d2[4 * q + 0], acc);
                acc = fmaf(w.y, d2[4 * q + 1], acc);
                acc = fmaf(w.z, d2[4 * q + 2], acc);
                acc = fmaf(w.w, d2[4 * q + 3], acc);
            }
            const float z = a1[k];
            o1[k] = acc * (1.f - z * z);
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0 && lsum != 0.f) {
        atomicAdd(loss, lsum / ((float)n * (float)O));
        if (n_epoch > 0) atomicAdd(loss + 1, lsum / ((float)n_epoch * (float)O));
    }
}

// Weight gradient as a reduction over samples: out[r][c] = sum_s D[s][r] A[s][c]
// for c < Cc, and the bias gradient out[r][Cc] = sum_s D[s][r] (a column of ones).
// 64x64 output tile per 256-thread block (4x4 per thread), samples in slices of
// kGK staged in shared memory; blockIdx.z takes a contiguous share of the
// samples and writes its own partial tile (summed in split order below).
__global__ void __launch_bounds__(256) wgrad_kernel(int64_t n, int R, int Cc, const float *__restrict__ D,
                                                    const float *__restrict__ A, int64_t per_split,
                                                    float *__restrict__ part)
{
    __shared__ __align__(16) float Ds[kGK][kGT];
    __shared__ __align__(16) float As[kGK][kGT];
    const int r0 = blockIdx.y * kGT, c0 = blockIdx.x * kGT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t sb = (int64_t)blockIdx.z * per_split, se = min((int64_t)n, sb + per_split);
    float acc[4][4] = {};
    for (int64_t s0 = sb; s0 < se; s0 += kGK) {
        for (int e = threadIdx.x; e < kGK * kGT; e += blockDim.x) {
            const int kk = e / kGT, j = e - kk * kGT;
            const int64_t s = s0 + kk;
            const bool in = s < se;
            Ds[kk][j] = (in && r0 + j < R) ? D[(size_t)s * R + r0 + j] : 0.f;
            const int c = c0 + j;
            As[kk][j] = !in ? 0.f : (c < Cc ? A[(size_t)s * Cc + c] : (c == Cc ? 1.f : 0.f));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            const float4 d = *reinterpret_cast<const float4 *>(&Ds[kk][4 * ty]);
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][4 * tx]);
            const float dv[4] = {d.x, d.y, d.z, d.w}, av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], av[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int W = Cc + 1;
    float *out = part + (size_t)blockIdx.z * R * W;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * ty + i;
        if (r >= R) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + 4 * tx + j;
            if (c < W) out[(size_t)r * W + c] = acc[i][j];
        }
    }
}

// dW[r][c] = sum over splits (in order) of part[z][r][c] for c < Cc; db[r] from column Cc.
__global__ void wgrad_reduce_kernel(int splits, int R, int Cc, const float *__restrict__ part, float *__restrict__ dW,
                                    float *__restrict__ db)
{
    const int W = Cc + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * W; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * R * W + e];
        const int r = (int)(e / W), c = (int)(e - (int64_t)r * W);
        if (c < Cc) dW[(size_t)r * Cc + c] = s;
        else db[r] = s;
    }
}

// Adam (decay rates b1, b2; c1 = 1 - b1^t, c2 = 1 - b2^t the bias corrections) on the
// FP32 master parameters.
__global__ void adam_kernel(size_t np, float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                            const float *__restrict__ Gr, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const float g = Gr[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// BF16 copy (round to nearest even) of W1 -> W1^T, W2 -> W2^T, W3.
__global__ void pack_bf16_kernel(int I, int H, int O, const float *__restrict__ P, __nv_bfloat16 *__restrict__ wb)
{
    const size_t n1 = (size_t)I * H, n2 = (size_t)H * H, n3 = (size_t)O * H;
    const size_t oW2 = n1 + H, oW3 = oW2 + n2 + H;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n1 + n2 + n3; k += (size_t)gridDim.x * blockDim.x) {
        size_t src;
        if (k < n1) {
            const size_t kk = k / H, j = k - kk * H;  // W1^T[kk][j] = W1[j][kk]
            src = j * I + kk;
        } else if (k < n1 + n2) {
            const size_t e = k - n1, kk = e / H, j = e - kk * H;
            src = oW2 + j * H + kk;
        } else {
            src = oW3 + (k - n1 - n2);
        }
        wb[k] = __float2bfloat16_rn(P[src]);
    }
}

// Xb[i] = X[perm[i]] (standardised when xm is given), Tb[i] = T[perm[i]] (and Wb[i] = Wt[perm[i]]
// with weights) for i < nn.
__global__ void gather_kernel(int64_t nn, int I, int O, const int64_t *__restrict__ perm, const float *__restrict__ X,
                              const float *__restrict__ T, const float *__restrict__ Wt, const float *__restrict__ xm,
                              const float *__restrict__ xinv, float *__restrict__ Xb, float *__restrict__ Tb,
                              float *__restrict__ Wb)
{
    const int64_t tot = nn * (I + O);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nn * I) {
            const int64_t i = e / I, k = e - i * I;
            const float x = X[(size_t)perm[i] * I + k];
            Xb[e] = xm ? (x - xm[k]) * xinv[k] : x;
        } else {
            const int64_t f = e - nn * I, i = f / O, k = f - i * O;
            Tb[f] = T[(size_t)perm[i] * O + k];
            if (Wt) Wb[f] = Wt[(size_t)perm[i] * O + k];
        }
    }
}

// phi0[c][g][i] = shrink max(exp(min(mu + sd y[c][g], t_cap)) - 1e-6, 0) at the 4 nodes (inverse of
// the target map, capped at the largest training target, times a shrink factor).
__global__ void predict_phi_kernel(int64_t CG, const float *__restrict__ Y, float mu, float sd, float t_cap,
                                   float shrink, double *__restrict__ phi)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < CG; e += (int64_t)gridDim.x * blockDim.x) {
        const double t = fmin((double)mu + (double)sd * (double)Y[e], (double)t_cap);
        const double v = (double)shrink * fmax(exp(t) - 1e-6, 0.0);
        double2 *o = reinterpret_cast<double2 *>(phi + (size_t)e * 4);
        o[0] = make_double2(v, v);
        o[1] = make_double2(v, v);
    }
}

Mlp *as_mlp(tf_handle h)
{
    auto *o = reinterpret_cast<Object *>(h);
    return (o && o->kind == Kind::Mlp) ? static_cast<Mlp *>(o) : nullptr;
}

int grid_for(int64_t work, int per_block, int cap)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, cap));
}

size_t fwd_smem(const Mlp &m)
{
    return sizeof(float) * ((size_t)kKC * m.H + (size_t)m.H * m.H + (size_t)m.O * m.H + 2 * m.H + m.O);
}
size_t bwd_smem(const Mlp &m) { return sizeof(float) * ((size_t)m.H * m.H + (size_t)m.O * m.H); }

// raw = true: X holds raw features (standardised on load when the handle has an input scale).
void launch_forward(const Mlp &m, int64_t n, const float *X, bool raw, float *Y, float *A1, float *A2, cudaStream_t st)
{
    const int blocks = (int)((n + 127) / 128);
    const size_t sm = fwd_smem(m);
    const float *xm = raw ? m.xm : nullptr, *xi = raw ? m.xinv : nullptr;
    switch (m.H) {
    case 8: forward_kernel<8><<<blocks, 128, sm, st>>>(n, m.I, m.O, m.wb, m.p, X, xm, xi, Y, A1, A2); break;
    case 16: forward_kernel<16><<<blocks, 128, sm, st>>>(n, m.I, m.O, m.wb, m.p, X, xm, xi, Y, A1, A2); break;
    case 32: forward_kernel<32><<<blocks, 128, sm, st>>>(n, m.I, m.O, m.wb, m.p, X, xm, xi, Y, A1, A2); break;
    default: forward_kernel<64><<<blocks, 128, sm, st>>>(n, m.I, m.O, m.wb, m.p, X, xm, xi, Y, A1, A2); break;
    }
}

void launch_backward(const Mlp &m, int64_t n, const float *Y, const float *T, const float *Wt, const float *A1,
                     const float *A2, float *DY, float *D1, float *D2, int64_t n_epoch, cudaStream_t st)
{
    const int blocks = (int)((n + 127) / 128);
    const size_t sm = bwd_smem(m);
    const float is = 1.f / m.sd;
#define TF_BWD(HH) \
    backward_kernel<HH><<<blocks, 128, sm, st>>>(n, m.I, m.O, m.wb, Y, T, Wt, m.mu, is, m.kappa, A1, A2, DY, D1, D2, m.loss, \
                                                 n_epoch)
    switch (m.H) {
    case 8: TF_BWD(8); break;
    case 16: TF_BWD(16); break;
    case 32: TF_BWD(32); break;
    default: TF_BWD(64); break;
    }
#undef TF_BWD
}

int splits_for(int64_t n, int R, int Cc)
{
    const int64_t tiles = (int64_t)((Cc + 1 + kGT - 1) / kGT) * ((R + kGT - 1) / kGT);
    const int64_t want = (2 * 152 + tiles - 1) / tiles;
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)kMaxSplits, (n + kGK - 1) / kGK}));
}

void launch_wgrad(Mlp &m, int64_t n, int R, int Cc, const float *D, const float *A, float *dW, float *db, cudaStream_t st)
{
    const int splits = splits_for(n, R, Cc);
    int64_t per = (n + splits - 1) / splits;
    per = (per + kGK - 1) / kGK * kGK;
    const dim3 grid((Cc + 1 + kGT - 1) / kGT, (R + kGT - 1) / kGT, splits);
    wgrad_kernel<<<grid, 256, 0, st>>>(n, R, Cc, D, A, per, m.part);
    const int64_t tot = (int64_t)R * (Cc + 1);
    wgrad_reduce_kernel<<<grid_for(tot, 256, 4096), 256, 0, st>>>(splits, R, Cc, m.part, dW, db);
}

tf_status ensure_scratch(Mlp &m, int64_t n)
{
    if ((size_t)n > m.act_cap) {
        cudaFree(m.act);
        m.act = nullptr;
        m.act_cap = 0;
        MLP_CUDA(cudaMalloc(&m.act, sizeof(float) * (size_t)n * (4 * m.H + 2 * m.O)));
        m.act_cap = (size_t)n;
    }
    if (!m.part) {
        // the largest partial-sum block any of the three layers can need
        const size_t need = (size_t)kMaxSplits * std::max({(size_t)m.H * (m.I + 1), (size_t)m.H * (m.H + 1),
                                                           (size_t)m.O * (m.H + 1)});
        MLP_CUDA(cudaMalloc(&m.part, sizeof(float) * need));
    }
    return TF_OK;
}

// Forward and backward over n samples: the gradient into m.g and the loss into m.loss[0].
// raw = true: X holds raw features, standardised first into scratch when the handle has
// an input scale (the first layer's weight gradient needs the standardised inputs).
tf_status gradients(Mlp &m, const float *X, bool raw, const float *T, const float *Wt, int64_t n, int64_t n_epoch,
                    cudaStream_t st)
{
    tf_status s = ensure_scratch(m, n);
    if (s != TF_OK) return s;
    if (raw && m.xm) {
        if ((size_t)n > m.xn_cap) {
            cudaFree(m.xn);
            m.xn = nullptr;
            m.xn_cap = 0;
            MLP_CUDA(cudaMalloc(&m.xn, sizeof(float) * (size_t)n * m.I));
            m.xn_cap = (size_t)n;
        }
        normalize_kernel<<<grid_for(n * m.I, 256, 8 * 152), 256, 0, st>>>(n, m.I, X, m.xm, m.xinv, m.xn);
        X = m.xn;
    }
    float *A1 = m.act, *A2 = A1 + (size_t)n * m.H, *D1 = A2 + (size_t)n * m.H, *D2 = D1 + (size_t)n * m.H;
    float *Y = D2 + (size_t)n * m.H, *DY = Y + (size_t)n * m.O;
    launch_forward(m, n, X, false, Y, A1, A2, st);
    MLP_CUDA(cudaMemsetAsync(m.loss, 0, sizeof(float), st));
    launch_backward(m, n, Y, T, Wt, A1, A2, DY, D1, D2, n_epoch, st);
    launch_wgrad(m, n, m.H, m.I, D1, X, m.g, m.g + m.off_b1(), st);
    launch_wgrad(m, n, m.H, m.H, D2, A1, m.g + m.off_W2(), m.g + m.off_b2(), st);
    launch_wgrad(m, n, m.O, m.H, DY, A2, m.g + m.off_W3(), m.g + m.off_b3(), st);
    MLP_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status repack(Mlp &m, cudaStream_t st)
{
    pack_bf16_kernel<<<grid_for((int64_t)m.np, 256, 2048), 256, 0, st>>>(m.I, m.H, m.O, m.p, m.wb);
    MLP_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status adam(Mlp &m, float lr, cudaStream_t st)
{
    ++m.step;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)m.step)), c2 = (float)(1.0 - std::pow(b2, (double)m.step));
    adam_kernel<<<grid_for((int64_t)m.np, 256, 2048), 256, 0, st>>>(m.np, m.p, m.m, m.v, m.g, lr, (float)b1, (float)b2,
                                                                    1e-8f, c1, c2);
    return repack(m, st);
}

}  // namespace

}  // namespace tf

using namespace tf;

extern "C" {

tf_status tf_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, tf_handle *out)
{
    if (!out) return fail(TF_ERR_ARG, "tf_mlp_create: out is NULL");
    *out = nullptr;
    if (n_in < 1 || !(n_hidden == 8 || n_hidden == 16 || n_hidden == 32 || n_hidden == 64) || n_out < 1 ||
        n_out > kMaxO)
        return fail(TF_ERR_ARG, "tf_mlp_create: need n_in >= 1, n_hidden in {8, 16, 32, 64}, 1 <= n_out <= 64");
    Mlp *m = new (std::nothrow) Mlp();
    if (!m) return fail(TF_ERR_NOMEM, "tf_mlp_create: allocation failed");
    m->I = n_in;
    m->H = n_hidden;
    m->O = n_out;
    m->np = (size_t)n_hidden * n_in + n_hidden + (size_t)n_hidden * n_hidden + n_hidden + (size_t)n_out * n_hidden + n_out;
    cudaGetDevice(&m->device);
    // Glorot-uniform weights, zero biases, from a seeded Mersenne twister on the host
    std::vector<float> p(m->np, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](size_t off, int fan_out, int fan_in) {
        const float a = std::sqrt(6.f / (float)(fan_in + fan_out));
        std::uniform_real_distribution<float> U(-a, a);
        for (size_t k = 0; k < (size_t)fan_out * fan_in; ++k) p[off + k] = U(rng);
    };
    fill(0, m->H, m->I);
    fill(m->off_W2(), m->H, m->H);
    fill(m->off_W3(), m->O, m->H);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->p, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * m->np);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->red, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m->p, p.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->g, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->loss, 0, 2 * sizeof(float));
    if (e == cudaSuccess) {
        pack_bf16_kernel<<<grid_for((int64_t)m->np, 256, 2048), 256>>>(m->I, m->H, m->O, m->p, m->wb);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        release(m);
        return fail(e == cudaErrorMemoryAllocation ? TF_ERR_NOMEM : TF_ERR_CUDA,
                    std::string("tf_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = reinterpret_cast<tf_handle>(static_cast<Object *>(m));
    return TF_OK;
}

tf_status tf_mlp_params(tf_handle h, float *get, const float *set, int64_t *n_params)
{
    Mlp *m = as_mlp(h);
    if (!m) return fail(TF_ERR_ARG, "tf_mlp_params: not a network handle");
    if (n_params) *n_params = (int64_t)m->np;
    if (!get && !set) return TF_OK;
    MLP_CUDA(cudaSetDevice(m->device));
    if (set) {
        MLP_CUDA(cudaMemcpy(m->p, set, sizeof(float) * m->np, cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemset(m->m, 0, sizeof(float) * m->np));
        MLP_CUDA(cudaMemset(m->v, 0, sizeof(float) * m->np));
        m->step = 0;
        tf_status s = repack(*m, nullptr);
        if (s != TF_OK) return s;
        MLP_CUDA(cudaDeviceSynchronize());
    }
    if (get) MLP_CUDA(cudaMemcpy(get, m->p, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
    return TF_OK;
}

tf_status tf_mlp_scale(tf_handle h, float *mu_get, float *sd_get, const float *mu_set, const float *sd_set)
{
    Mlp *m = as_mlp(h);
    if (!m) return fail(TF_ERR_ARG, "tf_mlp_scale: not a network handle");
    if (sd_set && !(*sd_set > 0.f)) return fail(TF_ERR_ARG, "tf_mlp_scale: sd must be > 0");
    if (mu_set) m->mu = *mu_set;
    if (sd_set) m->sd = *sd_set;
    if (mu_get) *mu_get = m->mu;
    if (sd_get) *sd_get = m->sd;
    return TF_OK;
}

tf_status tf_mlp_limits(tf_handle h, float *kappa_get, float *cap_get, const float *kappa_set, const float *cap_set)
{
    Mlp *m = as_mlp(h);
    if (!m) return fail(TF_ERR_ARG, "tf_mlp_limits: not a network handle");
    if (kappa_set && !(*kappa_set > 0.f)) return fail(TF_ERR_ARG, "tf_mlp_limits: overshoot weight must be > 0");
    if (cap_set && std::isnan(*cap_set)) return fail(TF_ERR_ARG, "tf_mlp_limits: cap is NaN");
    if (kappa_set) m->kappa = *kappa_set;
    if (cap_set) m->t_cap = *cap_set;
    if (kappa_get) *kappa_get = m->kappa;
    if (cap_get) *cap_get = m->t_cap;
    return TF_OK;
}

tf_status tf_mlp_shrink(tf_handle h, float *get, const float *set)
{
    Mlp *m = as_mlp(h);
    if (!m) return fail(TF_ERR_ARG, "tf_mlp_shrink: not a network handle");
    if (set && !(*set >= 0.f && *set <= 1.f)) return fail(TF_ERR_ARG, "tf_mlp_shrink: factor must be in [0, 1]");
    if (set) m->shrink = *set;
    if (get) *get = m->shrink;
    return TF_OK;
}

tf_status tf_mlp_input_scale(tf_handle h, float *mean_get, float *inv_get, const float *mean_set, const float *inv_set)
{
    Mlp *m = as_mlp(h);
    if (!m || (!mean_set) != (!inv_set)) return fail(TF_ERR_ARG, "tf_mlp_input_scale: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    const size_t bytes = sizeof(float) * (size_t)m->I;
    if (mean_set) {
        if (!m->xm) MLP_CUDA(cudaMalloc(&m->xm, bytes));
        if (!m->xinv) MLP_CUDA(cudaMalloc(&m->xinv, bytes));
        MLP_CUDA(cudaMemcpy(m->xm, mean_set, bytes, cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemcpy(m->xinv, inv_set, bytes, cudaMemcpyHostToDevice));
    }
    if (mean_get || inv_get) {
        if (!m->xm) return fail(TF_ERR_ARG, "tf_mlp_input_scale: the network has no input scale");
        if (mean_get) MLP_CUDA(cudaMemcpy(mean_get, m->xm, bytes, cudaMemcpyDeviceToHost));
        if (inv_get) MLP_CUDA(cudaMemcpy(inv_get, m->xinv, bytes, cudaMemcpyDeviceToHost));
    }
    return TF_OK;
}

tf_status tf_mlp_fit_inputs(tf_handle h, const float *X, int64_t n, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !X || n < 2) return fail(TF_ERR_ARG, "tf_mlp_fit_inputs: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * (size_t)m->I;
    if (!m->xm) MLP_CUDA(cudaMalloc(&m->xm, bytes));
    if (!m->xinv) MLP_CUDA(cudaMalloc(&m->xinv, bytes));
    double *acc = nullptr;  // sum [I], squared deviations [I], FP64 mean [I]
    MLP_CUDA(cudaMalloc(&acc, 3 * sizeof(double) * (size_t)m->I));
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double) * (size_t)m->I, st);
    const int grid = (int)std::min<int64_t>(n, 4 * 152);
    const int sgrid = grid_for(m->I, 256, 64);
    if (e == cudaSuccess) {
        colsum_kernel<<<grid, 256, 0, st>>>(n, m->I, X, nullptr, 0, acc);
        colstat_kernel<<<sgrid, 256, 0, st>>>(m->I, n, acc, nullptr, acc + 2 * m->I, m->xm, m->xinv, 0);
        colsum_kernel<<<grid, 256, 0, st>>>(n, m->I, X, acc + 2 * m->I, 1, acc + m->I);
        colstat_kernel<<<sgrid, 256, 0, st>>>(m->I, n, nullptr, acc + m->I, nullptr, nullptr, m->xinv, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(acc);
    if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("tf_mlp_fit_inputs: ") + cudaGetErrorString(e));
    return TF_OK;
}

tf_status tf_mlp_fit_scale(tf_handle h, const float *T, int64_t n_values, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !T || n_values < 2) return fail(TF_ERR_ARG, "tf_mlp_fit_scale: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    double acc[2] = {0.0, 0.0};
    MLP_CUDA(cudaMemsetAsync(m->red, 0, 2 * sizeof(double), st));
    const int grid = grid_for(n_values, 256, 4 * 152);
    moment_kernel<<<grid, 256, 0, st>>>(n_values, T, 0.0, 0, m->red);
    MLP_CUDA(cudaMemcpyAsync(acc, m->red, sizeof(double), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    const double mu = acc[0] / (double)n_values;
    moment_kernel<<<grid, 256, 0, st>>>(n_values, T, mu, 1, m->red + 1);
    MLP_CUDA(cudaMemcpyAsync(acc + 1, m->red + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    const double sd = std::sqrt(acc[1] / (double)n_values);
    unsigned key = 0u;
    unsigned *kd = reinterpret_cast<unsigned *>(m->red);
    MLP_CUDA(cudaMemsetAsync(kd, 0, sizeof(unsigned), st));
    max_key_kernel<<<grid, 256, 0, st>>>(n_values, T, kd);
    MLP_CUDA(cudaMemcpyAsync(&key, kd, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    const unsigned bits = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
    float tmax;
    std::memcpy(&tmax, &bits, sizeof(float));
    m->mu = (float)mu;
    m->sd = sd > 0.0 ? (float)sd : 1.f;
    m->t_cap = tmax;
    return TF_OK;
}

tf_status tf_mlp_features(int64_t n_cells, int32_t n_groups, const int32_t *cell_material, const double *sigma_t,
                          const double *sigma_s, const double *Q, const int32_t *nbr, float *X, void *stream)
{
    if (n_cells < 1 || n_groups < 1 || !cell_material || !sigma_t || !sigma_s || !Q || !nbr || !X)
        return fail(TF_ERR_ARG, "tf_mlp_features: bad arguments");
    features_kernel<<<grid_for(n_cells, 4, 65535), dim3(32, 4), 0, (cudaStream_t)stream>>>(
        n_cells, n_groups, cell_material, sigma_t, sigma_s, Q, nbr, X, n_groups * n_groups + 4 * n_groups);
    MLP_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status tf_mlp_features_context(int64_t n_cells, int32_t n_groups, const int32_t *cell_material,
                                  const double *sigma_t, const double *sigma_s, const double *Q, const int32_t *nbr,
                                  int32_t n_scales, const int32_t *steps, float *X, void *stream)
{
    if (n_cells < 1 || n_groups < 1 || !cell_material || !sigma_t || !sigma_s || !Q || !nbr || !X || n_scales < 0 ||
        n_scales > 16 || (n_scales > 0 && !steps))
        return fail(TF_ERR_ARG, "tf_mlp_features_context: bad arguments");
    for (int k = 0; k < n_scales; ++k)
        if (steps[k] < 0 || steps[k] > 100000 || (k > 0 && steps[k] < steps[k - 1]))
            return fail(TF_ERR_ARG, "tf_mlp_features_context: steps must be ascending, in [0, 100000]");
    cudaStream_t st = (cudaStream_t)stream;
    const int G = n_groups, base = G * G + 4 * G, ld = base + 2 * G * n_scales;
    features_kernel<<<grid_for(n_cells, 4, 65535), dim3(32, 4), 0, st>>>(n_cells, G, cell_material, sigma_t, sigma_s,
                                                                       Q, nbr, X, ld);
    MLP_CUDA(cudaGetLastError());
    if (n_scales == 0) return TF_OK;
    const size_t CG = (size_t)n_cells * G;
    double *buf = nullptr;  // vq, vs and their ping-pong copies
    MLP_CUDA(cudaMallocAsync(&buf, 4 * CG * sizeof(double), st));
    double *vq = buf, *vs = buf + CG, *tq = buf + 2 * CG, *ts = buf + 3 * CG;
    const unsigned gb = (unsigned)grid_for((int64_t)CG, 256, 8 * 152);
    context_init_kernel<<<gb, 256, 0, st>>>(n_cells, G, cell_material, sigma_t, Q, vq, vs);
    int done = 0;
    for (int k = 0; k < n_scales; ++k) {
        for (; done < steps[k]; ++done) {
            smooth_kernel<<<gb, 256, 0, st>>>(n_cells, G, nbr, vq, tq);
            smooth_kernel<<<gb, 256, 0, st>>>(n_cells, G, nbr, vs, ts);
            std::swap(vq, tq);
            std::swap(vs, ts);
        }
        context_write_kernel<<<gb, 256, 0, st>>>(n_cells, G, ld, base + 2 * G * k, vq, vs, X);
    }
    cudaError_t e = cudaGetLastError();
    const cudaError_t ef = cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = ef;
    MLP_CUDA(e);
    return TF_OK;
}

tf_status tf_mlp_targets(int64_t n_cells, int32_t n_groups, const double *phi, float *T, void *stream)
{
    if (n_cells < 1 || n_groups < 1 || !phi || !T) return fail(TF_ERR_ARG, "tf_mlp_targets: bad arguments");
    const int64_t CG = n_cells * n_groups;
    targets_kernel<<<grid_for(CG, 256, 8 * 152), 256, 0, (cudaStream_t)stream>>>(CG, phi, T);
    MLP_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status tf_mlp_weights(int64_t n_cells, int32_t n_groups, const double *phi, float floor_w, float *W, void *stream)
{
    if (n_cells < 1 || n_groups < 1 || !phi || !W || !(floor_w >= 0.f))
        return fail(TF_ERR_ARG, "tf_mlp_weights: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *gmax = nullptr;
    MLP_CUDA(cudaMalloc(&gmax, sizeof(unsigned long long) * (size_t)n_groups));
    const int64_t CG = n_cells * n_groups;
    cudaError_t e = cudaMemsetAsync(gmax, 0, sizeof(unsigned long long) * (size_t)n_groups, st);
    if (e == cudaSuccess) {
        group_max_kernel<<<grid_for(CG, 256, 8 * 152), 256, 0, st>>>(n_cells, n_groups, phi, gmax);
        weights_kernel<<<grid_for(CG, 256, 8 * 152), 256, 0, st>>>(n_cells, n_groups, phi, gmax, floor_w, W);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(gmax);
    if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("tf_mlp_weights: ") + cudaGetErrorString(e));
    return TF_OK;
}

tf_status tf_mlp_forward(tf_handle h, const float *X, int64_t n, float *Y, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !X || !Y || n < 1) return fail(TF_ERR_ARG, "tf_mlp_forward: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    launch_forward(*m, n, X, true, Y, nullptr, nullptr, (cudaStream_t)stream);
    MLP_CUDA(cudaGetLastError());
    return TF_OK;
}

tf_status tf_mlp_gradients(tf_handle h, const float *X, const float *T, const float *W, int64_t n, float *grad,
                           float *loss, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !X || !T || n < 1) return fail(TF_ERR_ARG, "tf_mlp_gradients: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    tf_status s = gradients(*m, X, true, T, W, n, 0, st);
    if (s != TF_OK) return s;
    if (grad) MLP_CUDA(cudaMemcpyAsync(grad, m->g, sizeof(float) * m->np, cudaMemcpyDeviceToHost, st));
    if (loss) MLP_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    return TF_OK;
}

tf_status tf_mlp_adam_step(tf_handle h, float lr, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !(lr > 0.f)) return fail(TF_ERR_ARG, "tf_mlp_adam_step: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    tf_status s = adam(*m, lr, (cudaStream_t)stream);
    if (s != TF_OK) return s;
    MLP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TF_OK;
}

tf_status tf_mlp_train(tf_handle h, const float *X, const float *T, const float *W, int64_t n, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float *loss_history, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !X || !T || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
        return fail(TF_ERR_ARG, "tf_mlp_train: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t B = std::min<int64_t>(batch, n);
    float *Xb = nullptr, *Tb = nullptr, *Wb = nullptr;
    int64_t *perm_d = nullptr;
    auto cleanup = [&]() {
        cudaFree(Xb);
        cudaFree(Tb);
        cudaFree(Wb);
        cudaFree(perm_d);
    };
    cudaError_t e = cudaMalloc(&Xb, sizeof(float) * (size_t)B * m->I);
    if (e == cudaSuccess) e = cudaMalloc(&Tb, sizeof(float) * (size_t)B * m->O);
    if (e == cudaSuccess && W) e = cudaMalloc(&Wb, sizeof(float) * (size_t)B * m->O);
    if (e == cudaSuccess) e = cudaMalloc(&perm_d, sizeof(int64_t) * (size_t)n);
    if (e != cudaSuccess) {
        cleanup();
        return fail(TF_ERR_NOMEM, std::string("tf_mlp_train: ") + cudaGetErrorString(e));
    }
    // minibatches are consecutive slices of a per-epoch shuffle (seeded Mersenne twister)
    std::vector<int64_t> perm(n);
    std::iota(perm.begin(), perm.end(), (int64_t)0);
    std::mt19937_64 rng(seed);
    tf_status s = TF_OK;
    for (int ep = 0; ep < epochs && s == TF_OK; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(perm_d, perm.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->loss + 1, 0, sizeof(float), st);
        for (int64_t b0 = 0; b0 < n && s == TF_OK && e == cudaSuccess; b0 += B) {
            const int64_t nn = std::min<int64_t>(B, n - b0);
            gather_kernel<<<grid_for(nn * (m->I + m->O), 256, 8 * 152), 256, 0, st>>>(nn, m->I, m->O, perm_d + b0, X, T,
                                                                                      W, m->xm, m->xinv, Xb, Tb, Wb);
            s = gradients(*m, Xb, false, Tb, Wb, nn, n, st);
            if (s == TF_OK) s = adam(*m, lr, st);
        }
        float l = 0.f;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->loss + 1, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && s == TF_OK) s = fail(TF_ERR_CUDA, std::string("tf_mlp_train: ") + cudaGetErrorString(e));
        if (loss_history) loss_history[ep] = l;
    }
    cleanup();
    return s;
}

tf_status tf_mlp_predict_phi(tf_handle h, const float *X, int64_t n_cells, double *phi, void *stream)
{
    Mlp *m = as_mlp(h);
    if (!m || !X || !phi || n_cells < 1) return fail(TF_ERR_ARG, "tf_mlp_predict_phi: bad arguments");
    MLP_CUDA(cudaSetDevice(m->device));
    cudaStream_t st = (cudaStream_t)stream;
    float *Y = nullptr;
    MLP_CUDA(cudaMalloc(&Y, sizeof(float) * (size_t)n_cells * m->O));
    launch_forward(*m, n_cells, X, true, Y, nullptr, nullptr, st);
    const int64_t CG = n_cells * m->O;
    predict_phi_kernel<<<grid_for(CG, 256, 8 * 152), 256, 0, st>>>(CG, Y, m->mu, m->sd, m->t_cap, m->shrink, phi);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(Y);
    if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("tf_mlp_predict_phi: ") + cudaGetErrorString(e));
    return TF_OK;
}

}  // extern "C"
