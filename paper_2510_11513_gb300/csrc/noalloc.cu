// Per-group flux statistics of a scalar-flux array without any device
// allocation: the reduction scratch is a file-scope __device__ array.
//
// Some callers cannot allocate device memory: a host program whose device
// memory is owned entirely by another runtime's pool (a cudaMalloc there fails
// or breaks that pool's accounting), or a latency-critical loop that must not
// pay cudaMalloc's implicit device-wide synchronisation.  They pass their own
// input and output buffers; the partial sums live in g_flux_scratch, which
// every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "tf_internal.h"

namespace tf {

namespace {

// 2^20 doubles (8 MiB): partials [blocks][n_groups][3]; at n_groups = 1024 it
// still holds 341 blocks.
constexpr size_t kScratchDoubles = size_t(1) << 20;
constexpr int kMaxGroups = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_flux_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};  // device address of g_flux_scratch, per device
int g_sm_count[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // the context that address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (the library does not link libcuda)
PFN_cuCtxGetCurrent_v4000 ctx_getter()
{
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

CUcontext current_ctx()
{
    CUcontext c = nullptr;
    PFN_cuCtxGetCurrent_v4000 fn = ctx_getter();
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

// The address a kernel on device `dev` uses for caller buffer p (device, managed, or page-locked
// host memory mapped into the device's address space); TF_ERR_ARG for memory the device cannot
// reach (plain pageable host memory) or an address not aligned to `align` bytes.
tf_status device_view(const void *p, size_t align, int dev, const char *name, const void **out)
{
    const std::string what = std::string("tf_integrated_flux_noalloc: ") + name;
    if ((uintptr_t)p % align) return fail(TF_ERR_ARG, what + " is not " + std::to_string(align) + "-byte aligned");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(TF_ERR_ARG, what + ": not memory the device can reach");
    }
    switch (at.type) {
    case cudaMemoryTypeDevice:
        if (at.device != dev) return fail(TF_ERR_ARG, what + " lives on another device");
        *out = p;
        break;
    case cudaMemoryTypeManaged:
        *out = p;
        break;
    case cudaMemoryTypeHost:
        if (!at.devicePointer) return fail(TF_ERR_ARG, what + ": page-locked host memory not mapped into the device");
        *out = at.devicePointer;
        break;
    default:
        return fail(TF_ERR_ARG, what + ": pageable host memory (pass device, managed or mapped page-locked memory)");
    }
    if ((uintptr_t)*out % align) return fail(TF_ERR_ARG, what + " is not " + std::to_string(align) + "-byte aligned");
    return TF_OK;
}

// Same reduction as the library's statistics kernel, with the cell volume
// given directly (V/4 is formed here, exactly, as 0.25 V).
__global__ void __launch_bounds__(256) flux_stats_kernel(const double *__restrict__ phi, const double *__restrict__ vol,
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
                iv += (0.25 * vol[c]) * s;
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

__global__ void flux_finish_kernel(const double *__restrict__ part, int nblk, int G, double *__restrict__ out)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        double m = 0.0, a = 0.0, b = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const double *p = part + ((size_t)k * G + g) * 3;
            m = fmax(m, p[0]);
            a += p[1];
            b += p[2];
        }
        out[3 * g + 0] = m;
        out[3 * g + 1] = a;
        out[3 * g + 2] = b;
    }
}

}  // namespace

}  // namespace tf

using namespace tf;

extern "C" tf_status tf_integrated_flux_noalloc(const double *phi, const double *volume, int64_t n_cells,
                                                int32_t n_groups, double *out, void *stream)
{
    if (!phi || !volume || !out || n_cells < 1)
        return fail(TF_ERR_ARG, "tf_integrated_flux_noalloc: NULL buffer or no cells");
    if (n_groups < 1 || n_groups > kMaxGroups)
        return fail(TF_ERR_ARG, "tf_integrated_flux_noalloc: n_groups must be in [1, " + std::to_string(kMaxGroups) +
                                    "]; the fixed scratch array is sized for at most that many groups");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TF_ERR_ARG, "tf_integrated_flux_noalloc: device ordinal too large");
    // the kernel reads phi as pairs of doubles (16 bytes), the volumes and the output as doubles
    const void *phi_d = nullptr, *vol_d = nullptr, *out_d = nullptr;
    tf_status s = device_view(phi, 16, dev, "phi", &phi_d);
    if (s == TF_OK) s = device_view(volume, 8, dev, "volume", &vol_d);
    if (s == TF_OK) s = device_view(out, 8, dev, "out", &out_d);
    if (s != TF_OK) return s;
    double *scratch = nullptr;
    int sms = 0;
    {
        // once per device and context, with that device current: the device address of the
        // scratch array (looked up again when the device's context changed, e.g. after a reset)
        std::lock_guard<std::mutex> lk(g_mu);
        const CUcontext ctx = current_ctx();
        if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_flux_scratch);
            if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double *>(p);
            g_sm_count[dev] = n;
            g_scratch_ctx[dev] = current_ctx();  // the lookup made the device's context current
        }
        scratch = g_scratch_addr[dev];
        sms = g_sm_count[dev];
    }
    int64_t nblk = std::min<int64_t>(4 * (int64_t)sms, (n_cells + 7) / 8);
    nblk = std::min<int64_t>(nblk, (int64_t)(kScratchDoubles / (3 * (size_t)n_groups)));
    if (nblk < 1) nblk = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every block overwrites its own [n_groups][3] slice, so nothing has to start at zero
    flux_stats_kernel<<<(unsigned)nblk, dim3(32, 8), 0, st>>>(static_cast<const double *>(phi_d),
                                                                static_cast<const double *>(vol_d), n_cells, n_groups,
                                                                scratch);
    flux_finish_kernel<<<(n_groups + 127) / 128, 128, 0, st>>>(scratch, (int)nblk, n_groups,
                                                               const_cast<double *>(static_cast<const double *>(out_d)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TF_ERR_CUDA, std::string("tf_integrated_flux_noalloc launch: ") + cudaGetErrorString(e));
    return TF_OK;
}
