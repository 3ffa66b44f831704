// Internal declarations of the tfsweep library (host C++ and CUDA).
#pragma once

#include <atomic>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/tfsweep.h"

namespace tf {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
tf_status fail(tf_status s, const std::string &msg);

// ------------------------------------------------------------------ objects
enum class Kind : int32_t { Mesh = 1, Quad = 2, Problem = 3, Mlp = 4 };

struct Object {
    explicit Object(Kind k) : kind(k) {}
    virtual ~Object() = default;
    Kind kind;
    std::atomic<int32_t> refs{1};
};

// Host geometry of a mesh of tetrahedra (nf = 4) or trilinear hexahedra (nf = 6), FP64.
struct Mesh : Object {
    Mesh() : Object(Kind::Mesh) {}
    int64_t nc = 0, nv = 0;
    int32_t nf = 4;                 // faces per cell
    std::vector<double> xyz;        // [nv][3]
    std::vector<int32_t> tets;      // [nc][4]     (tetrahedra)
    std::vector<int32_t> hexes;     // [nc][8]     (hexahedra; local vertex a + 2b + 4c at reference corner (a, b, c))
    std::vector<double> vol;        // [nc]
    std::vector<double> grad;       // [nc][4][3]  gradient of basis b_j (tetrahedra)
    std::vector<double> normal;     // [nc][nf][3] area-weighted outward normal of face f (tetrahedra: opposite
                                    //             vertex f; hexahedra: integrated over the face xi_d = s, f = 2d + s)
    std::vector<int32_t> nbr;       // [nc][nf]
    std::vector<int8_t> nbr_face;   // [nc][nf]    face index of this face inside the neighbour
    std::vector<int8_t> nbr_node;   // tetrahedra: [nc][4][4] neighbour-local index of local vertex i on face f
                                    // (-1 if none); hexahedra: [nc][6][4] of face-local node k
    // hexahedral element integrals (exact): M = int b_i b_j, G[d] = int b_i d b_j/dx_d,
    // F[f][d][k][l] = int_f N_d b_k b_l over face-local nodes (N the outward area-vector density)
    std::vector<double> hmass;      // [nc][8][8]
    std::vector<double> hgrad;      // [nc][3][8][8]
    std::vector<double> hface;      // [nc][6][3][4][4]
};

struct Quad : Object {
    Quad() : Object(Kind::Quad) {}
    int32_t D = 0;
    std::vector<double> omega;  // [D][3]
    std::vector<double> w;      // [D]
};

tf_status build_mesh(int64_t nv, const double *xyz, int64_t nc, const int32_t *tets, Mesh &m);
tf_status build_hex_mesh(int64_t nv, const double *xyz, int64_t nc, const int32_t *hexes, Mesh &m);
// local vertex of face-local node k (0..3) of hexahedral face f (0..5)
int hex_face_node(int f, int k);
tf_status build_quadrature(int32_t n_polar, int32_t n_az, Quad &q);

// Per-direction sweep graph and cell-block tasks.
struct TaskGraph {
    int32_t D = 0;
    int32_t cells_per_task = 0;
    int32_t max_level = 0;
    std::vector<int32_t> dir_levels;       // [D] number of t-levels
    // tasks, direction-major: tasks of direction a are [dir_task_begin[a], dir_task_begin[a+1])
    std::vector<int64_t> dir_task_begin;   // [D+1]
    std::vector<uint32_t> task_cell_begin; // [T]   into cell_list
    std::vector<uint16_t> task_ncell;      // [T]
    std::vector<uint16_t> task_dir;        // [T]
    std::vector<int32_t> task_level;       // [T]
    std::vector<int32_t> task_indeg;       // [T]   distinct upwind tasks
    std::vector<int32_t> task_blevel;      // [T]   longest path (in t-levels) from the task to a sink
    std::vector<uint64_t> down_begin;      // [T+1] into down_list
    std::vector<uint32_t> down_list;       // downwind task ids (global)
    std::vector<uint32_t> cell_list;       // (cell << cell_shift) | inflow mask, [D * nc]
    int32_t cell_shift = 4;                // 4 for tetrahedra, 6 for hexahedra (one mask bit per face)
    bool patches = false;                  // spatial patches: a task's cells may depend on each other
    // lagged back edges (empty when there are none): per cell entry (lag mask << 26) | first
    // slot; per slot its direction and (cell << 3) | face; slots of direction a are
    // [lag_dir_begin[a], lag_dir_begin[a + 1])
    std::vector<uint32_t> cell_lag;        // [D * nc] or empty
    std::vector<uint32_t> lag_slots;       // [2 * n_slots]
    std::vector<int64_t> lag_dir_begin;    // [D + 1]
    int64_t n_lagged() const { return lag_dir_begin.empty() ? 0 : lag_dir_begin.back(); }
    int64_t T() const { return (int64_t)task_ncell.size(); }
};

// Spatial-patch tasks (graph.cpp): regions are boxes of `extent` mean cell sizes;
// inside a patch, a cell that depends on one of the `gap` cells listed just before
// it is avoided when possible.
struct TaskShape {
    double extent = 2.0;
    int32_t gap = 1;
};

// Task shape a problem with options o on mesh m with G groups gets (api.cpp).
tf_status task_shape_of(const tf_options &o, const Mesh &m, int32_t G, bool *patches, TaskShape *shape);
// Cells per task (*B in: the caller's cells_per_task, >= 0; out: the grain) and shape (api.cpp).
tf_status task_grain(const tf_options &o, const Mesh &m, int32_t G, int32_t *B, bool *patches, TaskShape *shape);

// Face classification and levels only (no tasks); returns TF_ERR_CYCLE on a cycle.
// lag (non-null, [D][nc]): break cycles by lagged back edges instead of failing.
tf_status classify_and_level(const Mesh &m, const Quad &q, uint8_t *inflow, int32_t *level, uint8_t *lag = nullptr);
tf_status build_task_graph(const Mesh &m, const Quad &q, int32_t cells_per_task, TaskGraph &g,
                           const TaskShape *shape = nullptr, bool lag_cycles = false);

struct DeviceState;  // defined in the CUDA part

struct tf_autotune_report {
    int32_t n_candidates = 0, chosen = 0, cached = 0, sample_directions = 0;
    int32_t candidates[8] = {0};
    double seconds[8] = {0};
    // kernel-variant knobs tuned after the grain (only those the caller left automatic)
    int32_t pairing = 0, staging = 0, window = 0, n_variants = 0;
};

// Exact tables of the third-order (twenty-node) element (p3_tables.cpp), per unit
// volume / area: p[i] = int phi_i, M = int phi_i phi_j, C[k] = int phi_i d phi_j / d lambda_k,
// for the face opposite vertex f: fn[f] its ten nodes (node order), F[f] = int_f phi_r phi_c,
// fav[f][r] = int_f phi_r.
struct P3Tables {
    double p[20];
    double M[400];
    double C[4][400];
    int fn[4][10];
    double F[4][100];
    double fav[4][10];
};
void p3_element_tables(P3Tables &t);
void p3_node_alpha(int i, int al[4]);

struct Problem : Object {
    Problem() : Object(Kind::Problem) {}
    ~Problem() override;
    Mesh *mesh = nullptr;
    Quad *quad = nullptr;
    tf_options opt{};
    int32_t G = 0, M = 0;
    bool has_S1 = false, has_inflow = false;
    TaskGraph graph;
    DeviceState *dev = nullptr;
    tf_stats stats{};
    tf_autotune_report tune;
    tf_reduce_fn reduce = nullptr;  // sum over partners (direction sharding), or NULL
    void *reduce_user = nullptr;
};

// Picks cells_per_task, then the kernel variant (groups per lane: pairing; shared-memory
// staging) and the octant window, by timed trial sweeps over a direction sample
// (autotune.cpp); the chosen knobs are returned in *rep and written to *opt_out.
tf_status autotune_cells_per_task(const Mesh &m, const Quad &q, int32_t G, int32_t M, const int32_t *cell_material,
                                  const double *sigma_t, const double *sigma_s, const double *Q, const tf_options &opt,
                                  int32_t *out, tf_autotune_report *rep);

void retain(Object *o);
void release(Object *o);

// CUDA side (sweep.cu)
tf_status device_create(Problem &p, const int32_t *cell_material, const double *sigma_t, const double *sigma_s,
                        const double *Q, const double *S1, const double *psi_inflow);
void device_destroy(Problem &p);
tf_status device_sweep(Problem &p, const double *phi_in, double *phi_out, void *stream);
tf_status device_iterate(Problem &p, double tol, int32_t max_iters, double *phi, tf_iter_info *info, void *stream);
tf_status device_psi(Problem &p, int32_t dir, void *out, void *stream);
// Batched problems in shared persistent launches (sweep.cu).  sweep_only: one
// transport step phi_in -> phi (no statistics).
tf_status device_batch_iterate(const tf_handle *problems, int32_t n, double tol, int32_t max_iters, double *const *phi,
                               tf_iter_info *info, bool sweep_only, const double *const *phi_in, void *stream);

}  // namespace tf
