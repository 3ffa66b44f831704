// Level-synchronous sweep kernel (sm_103a): the bulk-synchronous schedule of
// Sec. 2.1 run on the GPU, as the ablation of the many-task sweep.  Each task is
// executed by exactly the same local-solve code as in sweep_kernel; only the
// order differs: buckets of (octant, t-level) in sequence, a barrier after each.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "tf_internal.h"

namespace tf {

#include "sweep_kernel.cuh"
#include "bsp.h"

namespace {

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Device-wide barrier of a co-resident grid: every CTA adds one arrival and
// waits until `target` arrivals are counted.  The fence before the arrival
// releases the CTA's psi stores (ordered before it by __syncthreads); the
// acquiring load and the second __syncthreads make every CTA's stores visible
// to all threads after it.  The wait is bounded: on the limit, or when another
// CTA has recorded an error, it returns false in every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int target, Ctrl *ctrl,
                                             unsigned long long limit_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = 1;
        fence_acq_rel_gpu();
        atomicAdd(bar, 1u);
        if (ld_acquire_u32(bar) < target) {
            const unsigned long long t0 = globaltimer();
            for (;;) {
                __nanosleep(20);
                if (ld_acquire_u32(bar) >= target) break;
                if (ld_volatile(&ctrl->error)) {
                    r = 0;
                    break;
                }
                if (globaltimer() - t0 > limit_ns) {
                    atomicCAS(&ctrl->error, 0, (int)TF_ERR_TIMEOUT);
                    r = 0;
                    break;
                }
            }
        }
        ok = r;
    }
    __syncthreads();
    return ok != 0;
}

// One task with the kernel variant MODE (the dispatch of sweep_kernel).
template <class T, int MODE>
__device__ __forceinline__ bool exec_task(const SweepArgs<T> &A, unsigned task, int lane, unsigned char *wsm,
                                          uint64_t *bars, uint32_t &ph, unsigned long long *wacc)
{
    const uint4 ti = __ldg(A.task + task);
    const uint32_t dir = ti.y >> 16;
    const V4<T> om = ld_ro(A.omega + dir);
    const size_t psi_dir = (size_t)(dir - (uint32_t)A.dir_begin) * (size_t)A.C;
    if constexpr (MODE == 3) {
        return run_task_pairs(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, wacc);
    } else if constexpr (MODE == 2) {
        return run_task_staged_any(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, wacc);
    } else if constexpr (MODE == 4) {
        return run_task_staged_any<T, 2>(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, wacc);
    } else if constexpr (MODE == 1) {
        run_task_wide(A, ti, lane, om.x, om.y, om.z, psi_dir);
        return true;
    } else if constexpr (MODE == 5) {
        run_task_p2(A, ti, lane, om.x, om.y, om.z, psi_dir);
        return true;
    } else if constexpr (MODE == 6) {
        return run_task_p2_staged(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm, bars, ph, wacc);
    } else if constexpr (MODE == 7) {
        extern __shared__ __align__(128) unsigned char dsm[];
        run_task_p3(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm,
                    reinterpret_cast<const P3Dev<T> *>(dsm + (size_t)(blockDim.x >> 5) * A.warp_smem));
        return true;
    } else if constexpr (MODE == 8) {
        run_task_hex(A, ti, lane, om.x, om.y, om.z, psi_dir);
        return true;
    } else if constexpr (MODE == 9) {
        run_task_hex_shared(A, ti, lane, om.x, om.y, om.z, psi_dir, wsm);
        return true;
    } else {
        run_task_generic(A, ti, lane, om.x, om.y, om.z, psi_dir);
        return true;
    }
}

// Warps claim the tasks of the current bucket one at a time (an atomic index per
// bucket: a dynamically scheduled parallel loop) and execute them; a warp that
// finds the bucket exhausted waits at the grid barrier until every CTA has
// finished the bucket.  The time warps spend there is counted as wait time, the
// time executing tasks as busy time.
template <class T, int MODE>
__global__ void __launch_bounds__(128, MODE == 7 ? (sizeof(T) == 4 ? 3 : 2) : MODE == 5 ? 2 : MODE == 6 ? 3 : MODE == 4 ? 6 : MODE == 9 ? (sizeof(T) == 4 ? 4 : 2) : MODE == 8 ? (sizeof(T) == 4 ? 3 : 2) : (sizeof(T) == 4 ? 4 : 3))
    bsp_sweep_kernel(const SweepArgs<T> A, const BspArgs S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *wsm = dsm + (size_t)(threadIdx.x >> 5) * A.warp_smem;
    uint32_t ph = 0;
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + A.warp_smem - 48);
    if constexpr (MODE == 2 || MODE == 3 || MODE == 4 || MODE == 6) {
        if (lane == 0) {
            for (int b = 0; b < 6; ++b) mbar_init(&bars[b], 1);
            fence_proxy_async_shared();
        }
        __syncwarp();
    }
    if constexpr (MODE == 7) {  // third order: the element tables after the warps' regions
        p3_stage_tables<T>(A.p3tab, dsm + (size_t)(blockDim.x >> 5) * A.warp_smem);
        __syncthreads();
    }
    __shared__ unsigned long long wstat[8][4];  // barrier wait ns, busy ns, tasks, data-wait cycles
    unsigned long long *ws = wstat[threadIdx.x >> 5];
    if (lane < 4) ws[lane] = 0;
    __syncwarp();
    const unsigned long long t_start = globaltimer();
    bool alive = true;
    unsigned int n_bar = 0;
    for (int b = S.b_lo; b < S.b_hi; ++b) {
        const uint32_t p0 = __ldg(S.bucket + b), p1 = __ldg(S.bucket + b + 1);
        while (alive) {
            uint32_t pos = 0;
            if (lane == 0) pos = p0 + (uint32_t)atomicAdd(S.claim + b, 1);
            pos = __shfl_sync(FULL, pos, 0);
            if (pos >= p1) break;
            const unsigned task = __ldg(S.order + pos);
            unsigned long long tb = 0;
            if (lane == 0) tb = globaltimer();
            if (task < A.task_begin || task >= A.task_end) {
                if (lane == 0) atomicCAS(&A.ctrl->error, 0, (int)TF_ERR_DEVICE);
                alive = false;
                break;
            }
            const bool ok = exec_task<T, MODE>(A, task, lane, wsm, bars, ph, ws + 3);
            alive = __all_sync(FULL, ok);
            if (lane == 0) {
                ws[1] += globaltimer() - tb;
                ++ws[2];
            }
        }
        if (b + 1 < S.b_hi) {
            unsigned long long t0 = 0;
            if (lane == 0) t0 = globaltimer();
            ++n_bar;
            if (!grid_barrier(S.bar, n_bar * gridDim.x + (unsigned)S.extra, A.ctrl, A.wait_limit_ns)) break;
            if (lane == 0) ws[0] += globaltimer() - t0;
        }
    }
    const unsigned long long t_end = globaltimer();
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&A.ctrl->tasks_done, ws[2]);
        atomicAdd(&A.ctrl->wait_ns, ws[0]);
        atomicAdd(&A.ctrl->busy_ns, ws[1]);
        atomicAdd(&A.ctrl->data_wait_cycles, ws[3]);
        atomicMin(&A.ctrl->t_first, t_start);
        atomicMax(&A.ctrl->t_last, t_end);
    }
}

template <class T, int MODE>
cudaError_t launch_one(const SweepArgs<T> &A, const BspArgs &S, int grid, int block, size_t dyn, bool cooperative,
                       cudaStream_t st)
{
    if (!cooperative) {
        bsp_sweep_kernel<T, MODE><<<grid, block, dyn, st>>>(A, S);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bsp_sweep_kernel<T, MODE>, A, S);
}

}  // namespace

template <> const void *bsp_kernel_fn<float>(int mode)
{
    switch (mode) {
    case 9: return (const void *)bsp_sweep_kernel<float, 9>;
    case 8: return (const void *)bsp_sweep_kernel<float, 8>;
    case 7: return (const void *)bsp_sweep_kernel<float, 7>;
    case 6: return (const void *)bsp_sweep_kernel<float, 6>;
    case 5: return (const void *)bsp_sweep_kernel<float, 5>;
    case 4: return (const void *)bsp_sweep_kernel<float, 4>;
    case 3: return (const void *)bsp_sweep_kernel<float, 3>;
    case 2: return (const void *)bsp_sweep_kernel<float, 2>;
    case 1: return (const void *)bsp_sweep_kernel<float, 1>;
    default: return (const void *)bsp_sweep_kernel<float, 0>;
    }
}

template <> const void *bsp_kernel_fn<double>(int mode)
{
    switch (mode) {
    case 9: return (const void *)bsp_sweep_kernel<double, 9>;
    case 8: return (const void *)bsp_sweep_kernel<double, 8>;
    case 7: return (const void *)bsp_sweep_kernel<double, 7>;
    case 5: return (const void *)bsp_sweep_kernel<double, 5>;
    case 2: return (const void *)bsp_sweep_kernel<double, 2>;
    case 1: return (const void *)bsp_sweep_kernel<double, 1>;
    default: return (const void *)bsp_sweep_kernel<double, 0>;
    }
}

template <>
cudaError_t launch_bsp<float>(const SweepArgs<float> &A, const BspArgs &S, int mode, int grid, int block, size_t dyn,
                              bool cooperative, cudaStream_t st)
{
    switch (mode) {
    case 9: return launch_one<float, 9>(A, S, grid, block, dyn, cooperative, st);
    case 8: return launch_one<float, 8>(A, S, grid, block, dyn, cooperative, st);
    case 7: return launch_one<float, 7>(A, S, grid, block, dyn, cooperative, st);
    case 6: return launch_one<float, 6>(A, S, grid, block, dyn, cooperative, st);
    case 5: return launch_one<float, 5>(A, S, grid, block, dyn, cooperative, st);
    case 4: return launch_one<float, 4>(A, S, grid, block, dyn, cooperative, st);
    case 3: return launch_one<float, 3>(A, S, grid, block, dyn, cooperative, st);
    case 2: return launch_one<float, 2>(A, S, grid, block, dyn, cooperative, st);
    case 1: return launch_one<float, 1>(A, S, grid, block, dyn, cooperative, st);
    default: return launch_one<float, 0>(A, S, grid, block, dyn, cooperative, st);
    }
}

template <>
cudaError_t launch_bsp<double>(const SweepArgs<double> &A, const BspArgs &S, int mode, int grid, int block,
                               size_t dyn, bool cooperative, cudaStream_t st)
{
    switch (mode) {
    case 9: return launch_one<double, 9>(A, S, grid, block, dyn, cooperative, st);
    case 8: return launch_one<double, 8>(A, S, grid, block, dyn, cooperative, st);
    case 7: return launch_one<double, 7>(A, S, grid, block, dyn, cooperative, st);
    case 5: return launch_one<double, 5>(A, S, grid, block, dyn, cooperative, st);
    case 2: return launch_one<double, 2>(A, S, grid, block, dyn, cooperative, st);
    case 1: return launch_one<double, 1>(A, S, grid, block, dyn, cooperative, st);
    default: return launch_one<double, 0>(A, S, grid, block, dyn, cooperative, st);
    }
}

}  // namespace tf
