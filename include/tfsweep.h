/*
 * tfsweep — unstructured S_N transport sweep on one GB300 (sm_103a).
 *
 * C ABI of the library.  Every call returns a tf_status; no exception or C++
 * type crosses this boundary.  Handles are opaque and reference counted: a
 * problem keeps its mesh and quadrature alive.  Handles are not thread safe;
 * use one handle from one host thread at a time.
 *
 * The operations follow the problem statement of Elwood et al., "An
 * Asynchronous Many-Task Algorithm for Unstructured S_N Transport on Shared
 * Memory Systems":
 *   - Eq. (1): steady multigroup transport with a total cross section, an
 *     external source and (here isotropic) scattering;
 *   - Eq. (2): the scalar flux as the quadrature sum phi = sum_a w_a psi_a;
 *   - Sec. 2.1 / Algorithm 1: the sweep — each direction's cells are solved
 *     in dependency order, every group inside one element visit, with the
 *     upwind face fluxes handed to downwind cells;
 *   - Eq. (3): the integrated flux per group and in total.
 * Spatial discretisation: upwind discontinuous Galerkin with nodal basis
 * functions: linear, quadratic or cubic on tetrahedra (NB = 4, 10 or 20 unknowns
 * per cell, group and direction; tf_options.order) or trilinear on hexahedra
 * (NB = 8; tf_mesh_create_hex).
 *
 * Memory conventions:
 *   - creation inputs are host arrays; they are copied, the caller keeps them;
 *   - phi arrays passed to tf_sweep / tf_source_iterate are caller-owned,
 *     FP64, layout [n_cells][n_groups][NB] (linear tetrahedra: node i of cell c
 *     is local vertex i of tets[c]; the node orders of the other elements are
 *     given with tf_options.order and tf_mesh_create_hex); they may live in
 *     device memory or in host memory (page-locked
 *     host buffers mapped into the device address space, as cudaHostAlloc and
 *     torch's pin_memory give, are read and written by the kernels directly
 *     in tf_sweep; other host buffers are copied in and out inside the call);
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Device-side failures (a device wait that ran out, a bounds flag) are read
 * back when the call synchronises and returned as its status; the handle
 * stays usable.
 */
#ifndef TFSWEEP_H
#define TFSWEEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tf_obj *tf_handle;

typedef enum {
    TF_OK = 0,
    TF_ERR_ARG = 1,            /* bad argument: NULL pointer, size out of range, wrong handle kind */
    TF_ERR_MESH = 2,           /* inverted/degenerate tetrahedron, bad vertex index, face shared by >2 cells */
    TF_ERR_CYCLE = 3,          /* a direction's cell dependency graph has a cycle */
    TF_ERR_CUDA = 4,           /* a CUDA runtime call failed (message in tf_last_error()) */
    TF_ERR_NOMEM = 5,          /* host or device allocation failed */
    TF_ERR_TIMEOUT = 6,        /* a device wait exceeded tf_options.wait_limit_s; the kernel returned */
    TF_ERR_NOT_CONVERGED = 7,  /* tf_source_iterate reached max_iters above tol (phi is still returned) */
    TF_ERR_DEVICE = 8          /* the device reported an inconsistent task graph (a bounds flag) */
} tf_status;

typedef enum { TF_FP32 = 0, TF_FP64 = 1 } tf_precision;

/* How the sweep accumulates phi = sum_a w_a psi_a in FP32 mode.  In FP64 mode
 * the accumulation is always plain FP64 additions. */
typedef enum {
    TF_PHI_PAIR = 0,  /* error-free FP32 pair (TwoProd/TwoSum) accumulation, rounded once to FP64 */
    TF_PHI_DADD = 1   /* one FP64 multiply-add per direction and node */
} tf_phi_accumulate;

/* Task schedule of the sweep.  All run (cell block, direction) tasks with the same local solves, and
 * a solve reads only finished upwind rows, so all give bit-identical psi and phi: only the order of
 * the work (and the default task grain, see cells_per_task) differs.
 *   TF_SCHED_AMT         asynchronous many-task (Sec. 3, Algorithm 1): one persistent launch per
 *                        direction chunk; a task runs as soon as its upwind tasks are done
 *                        (dependency counters, device ready queue).
 *   TF_SCHED_BSP         bulk-synchronous (Sec. 2.1): per direction chunk, buckets of (octant,
 *                        t-level) with the buckets of an octant's directions merged (simultaneous
 *                        angles); octants in sequence, levels in order, the tasks of a bucket in
 *                        parallel, a device-wide barrier after every bucket; one cooperative
 *                        persistent launch per chunk.
 *   TF_SCHED_BSP_LAUNCH  the same buckets with one kernel launch per bucket (the launch boundary
 *                        is the barrier).
 * Batched calls (n > 1) run only TF_SCHED_AMT problems. */
typedef enum { TF_SCHED_AMT = 0, TF_SCHED_BSP = 1, TF_SCHED_BSP_LAUNCH = 2 } tf_schedule;

/* Which cells form one task of a direction.  Both shapes solve the same units with the same
 * arithmetic and give bit-identical psi and phi; they differ in the memory traffic and the
 * parallelism of the sweep.
 *   TF_TASK_LEVELS   up to cells_per_task cells of one t-level (cells that do not depend on each
 *                    other: the buckets of Sec. 2.1 cut into blocks).
 *   TF_TASK_PATCHES  spatial patches: the cells of one small box of space (patch_extent mean cell
 *                    sizes on an edge) that can run together, listed in dependency order, at most
 *                    cells_per_task (<= 64) of them.  A cell's upwind neighbour in the same patch
 *                    was solved moments before by the same warp, so its face trace comes from
 *                    the on-chip caches or registers instead of device memory.  Each direction's
 *                    patch graph is acyclic by construction (a patch's round counts the region
 *                    boundaries crossed on the longest upwind path).  Linear tetrahedra with
 *                    n_groups a multiple of 32 and TF_SCHED_AMT only (else TF_ERR_ARG). */
typedef enum { TF_TASK_AUTO = 0, TF_TASK_LEVELS = 1, TF_TASK_PATCHES = 2 } tf_task_shape;

typedef struct {
    int32_t precision;       /* tf_precision: arithmetic of local solves and psi storage (default TF_FP32) */
    int32_t device;          /* CUDA device ordinal (default 0) */
    int32_t cells_per_task;  /* cells of one t-level grouped into one task; 0 = automatic (about 1024 units
                              * and at most 64 cells; 256 units and 4 to 16 cells on the packed-pair path;
                              * a quarter of that, at least 2, with a bulk-synchronous schedule),
                              * -1 = autotuned for use on its own (wall time of trial sweeps over a
                              * direction sample), -2 = autotuned for batched use (busy time of the
                              * warps); the tuner then also tries, at the chosen grain, the other
                              * groups-per-lane variant (pairing), registers instead of staging and an
                              * octant window of 2, for each of those options left at 0; choices cached
                              * per (precision, order, schedule, groups, directions, log2 cells) */
    int32_t dir_chunk;       /* directions swept per persistent launch; 0 = as many as the memory budget allows */
    int32_t warps_per_cta;   /* persistent kernel CTA size in warps; 0 = automatic */
    int32_t ctas_per_sm;     /* persistent CTAs per SM; 0 = as many as are resident */
    double wait_limit_s;     /* a device wait gives up after this many seconds (default 10) */
    int32_t phi_accumulate;  /* tf_phi_accumulate (default TF_PHI_PAIR) */
    int32_t inject_stall;    /* fault injection for tests: 1 = every device wait runs out (TF_SCHED_AMT:
                              * no task is seeded; TF_SCHED_BSP: each barrier waits for one CTA more
                              * than the grid holds); not allowed with TF_SCHED_BSP_LAUNCH */
    double psi_budget_gb;    /* device memory allowed for the angular-flux store; 0 = 80 % of free memory */
    int32_t task_order;      /* 0 = FIFO ready queue, seeds longest-critical-path first, and of the tasks
                              * a warp makes ready it runs next the one with the longest chain of
                              * downwind tasks (a direction's critical path skips the queue);
                              * 1 = the same, but the warp runs next the first task it made ready */
    int32_t staging;         /* 0 = automatic: stage each cell's rows in shared memory with bulk
                              * asynchronous copies when n_groups is a multiple of 32 and they fit,
                              * two cells ahead per warp with six CTAs per SM in FP32, three in FP64;
                              * 1 = never (registers only); 2 = two stages (FP32); 3 = three stages */
    int32_t octant_window;   /* directions are admitted one octant at a time; this many octants are
                              * active at once (the next one enters when the oldest is half done);
                              * 0 = automatic (8: every direction from the start) */
    int32_t pairing;         /* FP32, even group count: solve two groups per lane with packed FP32x2
                              * arithmetic.  0 = automatic (when n_groups is not a multiple of 32),
                              * 1 = never, 2 = whenever n_groups is even */
    int32_t schedule;        /* tf_schedule: how the sweep orders its tasks (default TF_SCHED_AMT) */
    int32_t order;           /* finite-element order: 0 or 1 = linear (4 nodes per cell), 2 = quadratic
                              * (10 nodes: the 4 vertices, then the midpoints of the local edges (0,1) (0,2)
                              * (0,3) (1,2) (1,3) (2,3)), 3 = cubic (20 nodes: the vertices, two per edge in
                              * that edge order, first at (2/3, 1/3) along the edge, then the centres of the
                              * faces opposite vertices 0..3); Q and every phi buffer are
                              * [n_cells][n_groups][nodes].  Orders 2 and 3: vacuum boundaries and no S1
                              * (both NULL), no batching */
    int32_t keep_ready;      /* ready tasks a warp keeps on a private stack and runs next (most recent
                              * first) instead of queueing them; 0 = automatic (1), at most 4 */
    int32_t task_shape;      /* tf_task_shape: which cells form one task (the grain of Sec. 3.4).
                              * 0 = automatic: spatial patches for linear tetrahedra with n_groups a
                              * multiple of 32 (no packed group pairs) under TF_SCHED_AMT, whose
                              * kernel variants solve a task's cells one after another; t-level
                              * blocks otherwise */
    double residual_floor;   /* stopping-test denominator floor, as a fraction of the group's max |phi|:
                              * 1 (the default; 0 also means 1) = per-group max-norm relative change,
                              * 1e-10 = pointwise relative change (unreachable in FP32 where DG
                              * undershoots put |phi| near 0) */
    double patch_extent;     /* spatial patches: edge of a patch region in mean cell sizes (the edge of
                              * a cube of six tetrahedra of the mean volume); 0 = automatic (2) */
    int32_t lag_cycles;      /* 0 = a direction whose sweep graph has a cycle is an error (TF_ERR_CYCLE);
                              * 1 = break the cycles by lagged back edges (hexahedral meshes, t-level
                              * tasks, problems swept on their own): whenever no cell is ready, a walk
                              * from the lowest-numbered waiting cell across the lowest-numbered open
                              * inflow faces (upwind neighbour not yet reached) finds a cycle, and the
                              * face that closes it is lagged.  A lagged face reads the upwind cell's
                              * psi of the previous transport step (zero in the first step), so a
                              * transport step is no longer an exact inversion of the streaming
                              * operator; source iteration converges to the same answer.  The sweep
                              * graph with cycles is outside the paper, which assumes a DAG per angle
                              * (Sec. 1); the particle balance holds only at convergence. */
    int32_t reserved_i;
    double reserved_d[1];
} tf_options;

/* Fills *opt with the defaults above. */
void tf_options_default(tf_options *opt);

/* Per-problem result of tf_source_iterate. */
typedef struct {
    int32_t iterations;        /* sweeps performed */
    int32_t converged;         /* 1 if the stopping test fell below tol */
    double residual;           /* last value of the stopping test r (see tf_source_iterate) */
    double integrated_total;   /* Eq. (3): sum over groups of the integrated flux of the final phi */
    double *integrated_flux;   /* caller host array [n_groups] or NULL: per-group integral of phi over space */
    double *residual_history;  /* caller host array [max_iters] or NULL: residual after each sweep */
    double seconds;            /* batched calls: wall time from the call's start to this problem's
                                * convergence (or to the end) */
    double balance;            /* particle balance of the last transport step, FP64 on the device:
                                * max over groups of |leakage + absorption - source| / max(source,
                                * absorption), with leakage the boundary outflow minus prescribed
                                * inflow, absorption sum_c sigma_t int_c phi, source int (Q + scattering)
                                * as the sweep used it; zero up to rounding of the local solves */
} tf_iter_info;

/* Scheduling statistics of the last sweep of a problem (for measurement). */
typedef struct {
    int64_t n_tasks;           /* (cell block, direction) tasks per sweep */
    int64_t n_units;           /* cells x directions x groups */
    int32_t n_dirs;
    int32_t max_level;         /* longest dependency chain over directions (t-levels - 1) */
    int32_t n_chunks;          /* persistent launches per sweep */
    int32_t grid_ctas;         /* persistent CTAs per launch */
    int32_t warps_per_cta;
    int32_t cells_per_task;
    int64_t tasks_executed;    /* counted on the device in the last sweep */
    int64_t wait_polls;        /* device polls of an empty queue slot in the last sweep */
    double wait_seconds;       /* summed over warps: time spent waiting for a ready task (TF_SCHED_AMT)
                                * or at the barriers between buckets (TF_SCHED_BSP) */
    double busy_seconds;       /* summed over warps: time spent executing tasks */
    double kernel_seconds;     /* first warp start to last warp end, summed over launches */
    double mean_ready;         /* mean ready-queue depth sampled at pops */
    /* CUDA-event times on the caller's stream (seconds): last transport step, and summed
     * over all steps since the problem was created (cum_steps of them) */
    double source_event_seconds, sweep_event_seconds, phi_event_seconds;
    double cum_source_event_seconds, cum_sweep_event_seconds, cum_phi_event_seconds;
    int64_t cum_steps;
    int64_t launches_per_step;  /* kernels this library launches per transport step */
    int32_t kernel_mode;        /* sweep kernel variant: 0 any G, 1 G%32==0 (registers), 2 G%32==0 staged
                                 * in shared memory (three stages), 3 packed group pairs (FP32, even G),
                                 * 4 G%32==0 staged, two stages, six CTAs per SM (FP32) */
    /* task-grain autotuning (cells_per_task < 0 at creation): candidate grains and the time
     * of one trial sweep over a direction sample for each; tuned_cached = 1 if the choice
     * came from an earlier problem of the same class */
    int32_t tuned_n, tuned_cached;
    int32_t tuned_candidates[8];
    double tuned_seconds[8];
    int32_t n_buckets;          /* bulk-synchronous schedules: (octant, t-level) buckets per sweep,
                                 * summed over direction chunks (barriers + chunks); 0 for TF_SCHED_AMT */
    /* autotuning: the kernel-variant knobs in use after it (tf_options.pairing, staging,
     * octant_window; 0 = automatic), tuned after the grain where the caller left them automatic */
    int32_t tuned_pairing, tuned_staging, tuned_window;
    int32_t task_shape;        /* tf_task_shape in use: TF_TASK_LEVELS or TF_TASK_PATCHES */
    double data_wait_seconds;  /* summed over warps: time waiting for rows staged by bulk copies
                                * (SM cycles at the nominal SM clock) */
    int64_t lagged_faces;      /* lagged back edges over all directions (lag_cycles) */
    double reserved_d[4];
} tf_stats;

/* Mesh of tetrahedra.  xyz: host [n_vertices][3] FP64; tets: host [n_cells][4]
 * vertex indices.  Tetrahedra must be positively oriented (det of the edge
 * vectors x1-x0, x2-x0, x3-x0 > 0) and conforming (a face is shared by at most
 * two cells).  Computes volumes, basis gradients (Table 1's f_i df_j/dx
 * ingredients), area-weighted outward face normals and face neighbours.
 * Host-only: no CUDA call.  Errors: TF_ERR_ARG, TF_ERR_MESH, TF_ERR_NOMEM. */
tf_status tf_mesh_create(int64_t n_vertices, const double *xyz, int64_t n_cells, const int32_t *tets,
                         tf_handle *out);

/* Mesh of trilinear hexahedra (the element of the paper's twisted hex grids, Sec. 2).
 * xyz: host [n_vertices][3] FP64; hexes: host [n_cells][8] vertex indices, local
 * vertex a + 2b + 4c at the corner (a, b, c) of the reference cube [0,1]^3 (so
 * 0-1, 0-2 and 0-4 are the edges at vertex 0).  The Jacobian determinant of the
 * trilinear map must be positive at the 27 points of the {0, 1/2, 1}^3 lattice; a
 * face (f = 2d + s, the reference face xi_d = s) is shared by at most two cells.
 * Computes, exactly (polynomial integration, FP64): volumes; mass int b_i b_j;
 * streaming int b_i d b_j / dx_d; face matrices int_f N_d b_k b_l over each face's
 * four nodes (N the outward area-vector density, non-planar faces included); the
 * integrated face area vectors (half the cross product of the face diagonals,
 * outward), which classify faces (inflow iff Omega.Nbar_f < -1e-12 |Nbar_f|); face
 * neighbours.  At most 2^26 - 1 cells.  Host-only: no CUDA call.
 * Errors: TF_ERR_ARG, TF_ERR_MESH, TF_ERR_NOMEM.  Problems on such a mesh take the
 * trilinear element (opt->order 0 or 1); their Q, phi and psi hold the eight vertex values
 * of every cell ([n_cells][n_groups][8]); S1 adds (Omega.S1) int b_i per node, and
 * psi_inflow is read at the vertices of boundary inflow faces. */
tf_status tf_mesh_create_hex(int64_t n_vertices, const double *xyz, int64_t n_cells, const int32_t *hexes,
                             tf_handle *out);

/* Element integrals of a hexahedral mesh (host outputs; any may be NULL):
 * mass [n_cells][8][8] = int b_i b_j; grad [n_cells][3][8][8] = int b_i d b_j / dx_d;
 * face [n_cells][6][3][4][4] = int_f N_d b_k b_l, k and l the face-local nodes (the
 * face's vertices in increasing local index).  Errors: TF_ERR_ARG (not a
 * hexahedral mesh). */
tf_status tf_mesh_hex_integrals(tf_handle mesh, double *mass, double *grad, double *face);

/* Angular quadrature.  Either a product rule (omega == NULL): n_polar
 * Gauss-Legendre cosines times n_azimuthal azimuths (k + 1/2) 2 pi / n_azimuthal,
 * weights summing to 4 pi, direction index a = polar * n_azimuthal + azimuth;
 * or explicit directions (omega != NULL): n_dirs unit vectors omega [n_dirs][3]
 * and weights w [n_dirs] (host FP64).  Directions are the S_N set of Eq. (2).
 * Host-only.  Errors: TF_ERR_ARG. */
tf_status tf_quadrature_create(int32_t n_polar, int32_t n_azimuthal, int32_t n_dirs, const double *omega,
                               const double *w, tf_handle *out);

/* Transport problem: mesh + quadrature + n_groups energy groups + materials
 * (Eq. (1)).  Host inputs, copied to the device selected by opt->device:
 *   cell_material [n_cells] in [0, n_materials);
 *   sigma_t [n_materials][n_groups] total cross section (> 0);
 *   sigma_s [n_materials][n_groups][n_groups], element [m][g_from][g_to];
 *   Q [n_cells][n_groups][NB] total isotropic volumetric source at the nodes
 *     (the angular source per steradian is (Q + sum_g' sigma_s phi_g') / 4 pi);
 *   S1 [n_cells][n_groups][3] or NULL: adds the angular source Omega . S1
 *     (constant per cell; used by manufactured-solution tests);
 *   psi_inflow [n_vertices][n_groups] or NULL: isotropic inflow prescribed at
 *     boundary vertices; NULL means vacuum boundaries.
 * Builds, per direction, the face classification (inflow iff Omega.N_f <
 * -1e-12 |N_f|), t-levels (Sec. 2.1), cell-block tasks and their dependency
 * counts (Sec. 3.5), and allocates the device state.  opt may be NULL.
 * Errors: TF_ERR_ARG, TF_ERR_CYCLE, TF_ERR_CUDA, TF_ERR_NOMEM. */
tf_status tf_problem_create(tf_handle mesh, tf_handle quad, int32_t n_groups, int32_t n_materials,
                            const int32_t *cell_material, const double *sigma_t, const double *sigma_s,
                            const double *Q, const double *S1, const double *psi_inflow, const tf_options *opt,
                            tf_handle *out);

/* One transport step per problem: source update q = (Q + sum_g' sigma_s phi_in)/4 pi,
 * a sweep of every direction (Algorithm 1: dependency counters released by
 * atomics, ready (cell block, direction) tasks pulled from a device queue),
 * and phi_out = sum_a w_a psi_a (Eq. 2).  phi_in / phi_out: [n] arrays of FP64
 * [n_cells][n_groups][NB] buffers (device or host); phi_in[k] may equal
 * phi_out[k].  Synchronises `stream` before returning.
 * Errors: TF_ERR_ARG, TF_ERR_CUDA, TF_ERR_TIMEOUT, TF_ERR_DEVICE. */
tf_status tf_sweep(const tf_handle *problems, int32_t n, const double *const *phi_in, double *const *phi_out,
                   void *stream);

/* Source iteration (group-Jacobi): repeat tf_sweep until the stopping test
 * r = max over (cell, group, node) of |phi_new - phi_old| / max(|phi_new|, f x max over the group of |phi_new|)
 * falls below tol or max_iters sweeps were done; f = opt.residual_floor (default 1: r is the largest
 * per-group max-norm relative change).  The difference and the denominator are FP64 on the device.
 * phi[k]: in = initial flux (NULL entry = zero start), out = final flux
 * (a NULL entry is not allowed for the output: pass a buffer).  info: [n] or
 * NULL.  Returns TF_ERR_NOT_CONVERGED if any problem stopped at max_iters.
 * Errors: as tf_sweep, plus TF_ERR_NOT_CONVERGED. */
tf_status tf_source_iterate(const tf_handle *problems, int32_t n, double tol, int32_t max_iters,
                            double *const *phi, tf_iter_info *info, void *stream);

/* Releases a handle (mesh, quadrature or problem).  Objects live until the last
 * problem that uses them is destroyed.  NULL is accepted. */
tf_status tf_destroy(tf_handle h);

/* ---------------------------------------------------------------- inspection */

/* Mesh geometry as computed by tf_mesh_create (host outputs; any may be NULL):
 * vol [n_cells]; normal [n_cells][4][3] area-weighted outward normal of the face
 * opposite local vertex f; nbr [n_cells][4] (-1 = boundary); nbr_node
 * [n_cells][4][4]: local index, in the neighbour across face f, of local vertex
 * i of the cell (-1 for i == f or a boundary face).  For a hexahedral mesh
 * (tf_mesh_create_hex): normal [n_cells][6][3] integrated outward area vectors;
 * nbr [n_cells][6]; nbr_node [n_cells][6][4]: local index, in the neighbour, of
 * face-local node k (-1 on the boundary). */
tf_status tf_mesh_geometry(tf_handle mesh, int64_t *n_cells, int64_t *n_vertices, double *vol, double *normal,
                           int32_t *nbr, int32_t *nbr_node);

/* Directions and weights of a quadrature (host outputs; any may be NULL). */
tf_status tf_quadrature_get(tf_handle quad, int32_t *n_dirs, double *omega, double *w);

/* Host-only: face classification and t-levels for every direction (Sec. 2.1
 * buckets), tetrahedral or hexahedral mesh.  inflow [n_dirs][n_cells]: bit f set iff face f is inflow;
 * level [n_dirs][n_cells].  Either may be NULL.  Errors: TF_ERR_CYCLE. */
tf_status tf_graph_levels(tf_handle mesh, tf_handle quad, uint8_t *inflow, int32_t *level);

/* Host-only: as tf_graph_levels, with cycles broken by lagged back edges (tf_options.lag_cycles):
 * lag [n_dirs][n_cells], bit f set iff inflow face f is lagged; levels count the other faces
 * only.  Either output may be NULL.  The paper has no counterpart (it assumes acyclic graphs).
 * Errors: TF_ERR_ARG. */
tf_status tf_graph_lag(tf_handle mesh, tf_handle quad, uint8_t *inflow, int32_t *level, uint8_t *lag);

/* Host-only: the tasks a problem with options *opt (NULL = defaults) and n_groups groups on this
 * mesh and quadrature would sweep (t-level blocks or spatial patches, tf_task_shape; the grain
 * and shape chosen as tf_problem_create chooses them, without the autotuner: a negative
 * cells_per_task is TF_ERR_ARG here).  *n_tasks: the number of tasks over all directions.
 * task_of [n_dirs][n_cells]: the task (0 .. n_tasks - 1) that solves each cell in each direction;
 * position [n_dirs][n_cells]: the cell's place in its task's list (a task solves its cells in
 * that order); indeg [n_tasks]: the number of distinct other tasks holding an upwind cell of the
 * task (its dependency counter's start).  Any array may be NULL (call once with all three NULL to
 * learn n_tasks).  Errors: TF_ERR_ARG, TF_ERR_CYCLE, TF_ERR_NOMEM. */
tf_status tf_graph_tasks(tf_handle mesh, tf_handle quad, const tf_options *opt, int32_t n_groups, int64_t *n_tasks,
                         int32_t *task_of, int32_t *position, int32_t *indeg);

/* Sum over the partners of a problem: replace buf[0 .. count) (device memory, FP64) by its
 * elementwise sum over every partner's buffer of the same call (for example an allreduce across
 * the processes that each sweep a share of the directions).  Called on the host thread of
 * tf_sweep / tf_source_iterate with the stream their work runs on: the reduction must be
 * enqueued on that stream (as an NCCL allreduce is) or finished before returning.  Return 0 on
 * success; anything else ends the call with TF_ERR_CUDA. */
typedef int32_t (*tf_reduce_fn)(void *user, double *buf, int64_t count, void *stream);

/* Direction sharding.  A problem whose quadrature holds a share of a direction set (explicit
 * omega and w in tf_quadrature_create) sweeps only those directions, so its phi = sum_a w_a psi_a
 * (Eq. (2)) is a partial sum.  With a reduce function set, every transport step hands that
 * partial phi ([n_cells][n_groups][NB] doubles) and this step's boundary leakage per group
 * (n_groups doubles, for the particle balance) to `fn` right after the phi reduction and before
 * the statistics, the stopping test and the next source update, so all partners iterate on the
 * same full phi and take the same stopping decision.  fn = NULL removes it.  A problem with a
 * reduce function runs its iterations without CUDA-graph capture and cannot be batched (n > 1:
 * TF_ERR_ARG).  Errors: TF_ERR_ARG. */
tf_status tf_problem_set_reduce(tf_handle problem, tf_reduce_fn fn, void *user);

/* Copies the angular flux of direction `dir` from the last sweep of `problem`
 * into out (device memory, [n_cells][n_groups][NB] in the problem precision:
 * float or double).  The direction must belong to the last direction chunk
 * swept (with one chunk: any direction).  Errors: TF_ERR_ARG, TF_ERR_CUDA. */
tf_status tf_problem_psi(tf_handle problem, int32_t dir, void *out, void *stream);

/* Scheduling statistics of the problem's last sweep. */
tf_status tf_problem_stats(tf_handle problem, tf_stats *out);

/* Per-group statistics of a scalar-flux array, computed without allocating any
 * device memory.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory, such as a host program whose device memory
 * is owned entirely by another runtime's pool, or a latency-critical loop that
 * must not pay cudaMalloc's implicit device synchronisation.
 *   phi    [n_cells][n_groups][4] FP64 nodal scalar flux, 16-byte aligned;
 *   volume [n_cells] FP64 cell volumes;
 *   out    [n_groups][3] FP64: max |phi|, sum_c (V_c/4) sum_i phi, and the
 *          plain nodal sum sum_c sum_i phi.
 * Each buffer must be memory the current device can reach: device memory of
 * that device, managed memory, or page-locked host memory mapped into the
 * device (cudaHostAlloc, torch's pin_memory); plain pageable host memory or a
 * misaligned address is refused with TF_ERR_ARG before anything is launched.
 * Runs on the current device, asynchronously on `stream`.  Its reduction
 * scratch is one fixed 8 MiB array per device (held by every GPU that loads
 * the library until the process exits), shared by all calls: calls that
 * overlap on the GPU race on it.  Each call overwrites the part it uses, so
 * nothing carries over between calls.  The first call on a device (and the
 * first after the device's context changed, e.g. after cudaDeviceReset) looks
 * the array up (cudaGetSymbolAddress); make that call before any stream
 * capture.  n_groups must be at most 1024 (TF_ERR_ARG otherwise).
 * Errors: TF_ERR_ARG, TF_ERR_CUDA. */
tf_status tf_integrated_flux_noalloc(const double *phi, const double *volume, int64_t n_cells, int32_t n_groups,
                                     double *out, void *stream);

/* Static description of a status code. */
const char *tf_status_string(tf_status s);

/* Detail of the last error on the calling thread ("" if none). */
const char *tf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TFSWEEP_H */
