// Level-synchronous (bulk-synchronous) sweep schedule: the scheme the paper's
// many-task sweep replaces (Sec. 2.1, Sec. 3; Fig. 2, centre).
// Included inside namespace tf after sweep_kernel.cuh (it needs SweepArgs).
#pragma once

// Buckets of one direction chunk: bucket b holds the tasks of every direction
// of one octant whose cells lie on one t-level (the buckets of an octant's
// directions merged level by level: simultaneous angles).  Buckets run in
// sequence (octants one after another, levels in increasing order), the tasks
// of one bucket in parallel, with a device-wide barrier after each bucket.
struct BspArgs {
    const uint32_t *order;   // task ids, grouped by bucket
    const uint32_t *bucket;  // [n_buckets + 1] offsets into order (global bucket index)
    int *claim;              // per bucket: tasks claimed so far (zero before the launch)
    unsigned int *bar;       // grid-barrier arrivals in this launch (zero before the launch)
    int32_t b_lo, b_hi;      // buckets run by this launch
    int32_t extra;           // fault injection for tests: 1 = every barrier waits for one arrival
                             // more than the grid has CTAs, so every wait runs out
};

// Kernel entry of a sweep-kernel variant (mode as in sweep_kernel), for
// occupancy queries and the dynamic shared-memory attribute.
template <class T> const void *bsp_kernel_fn(int mode);

// Launches buckets [S.b_lo, S.b_hi) of one chunk.  cooperative = one launch
// over several buckets with a grid barrier between them (the grid must be
// co-resident: at most the resident CTAs per SM x SMs); otherwise S must hold
// one bucket, and the kernel boundary is the barrier.
template <class T>
cudaError_t launch_bsp(const SweepArgs<T> &A, const BspArgs &S, int mode, int grid, int block, size_t dyn,
                       bool cooperative, cudaStream_t st);
