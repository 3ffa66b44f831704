// The C ABI: handle management, argument validation, error reporting.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "tf_internal.h"

namespace tf {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

tf_status fail(tf_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

void retain(Object *o)
{
    if (o) o->refs.fetch_add(1);
}

void release(Object *o)
{
    if (o && o->refs.fetch_sub(1) == 1) delete o;
}

Problem::~Problem()
{
    device_destroy(*this);
    release(mesh);
    release(quad);
}

namespace {

template <class T>
T *as(tf_handle h, Kind k)
{
    auto *o = reinterpret_cast<Object *>(h);
    if (!o || o->kind != k) return nullptr;
    return static_cast<T *>(o);
}

}  // namespace

}  // namespace tf

namespace tf {
// The kernel variants that solve a task's cells one after another (lanes over the groups of
// one cell: n_groups a multiple of 32, FP32 without packed group pairs or FP64) accept tasks
// whose cells depend on each other; the others, and the bulk-synchronous schedules (whose
// buckets are t-levels), take t-level blocks.
tf_status task_shape_of(const tf_options &o, const Mesh &m, int32_t G, bool *patches, TaskShape *shape)
{
    const bool paired = o.precision == TF_FP32 && G % 2 == 0 && (o.pairing == 2 || (o.pairing == 0 && G % 32 != 0));
    const bool ok = m.nf == 4 && o.order <= 1 && o.schedule == TF_SCHED_AMT && G % 32 == 0 && !paired;
    if (o.task_shape < TF_TASK_AUTO || o.task_shape > TF_TASK_PATCHES)
        return fail(TF_ERR_ARG, "task_shape must be a tf_task_shape");
    if (o.task_shape == TF_TASK_PATCHES && !ok)
        return fail(TF_ERR_ARG, "spatial patches need linear tetrahedra, n_groups a multiple of 32, no packed "
                                "group pairs and TF_SCHED_AMT");
    if (!(o.patch_extent >= 0.0) || o.patch_extent > 64.0)
        return fail(TF_ERR_ARG, "patch_extent must be in [0, 64]");
    *patches = o.task_shape == TF_TASK_PATCHES || (o.task_shape == TF_TASK_AUTO && ok);
    shape->extent = o.patch_extent > 0.0 ? o.patch_extent : 2.0;
    // the staged kernels issue a cell's copies one cell ahead (two stages) or two (three stages)
    const bool three = o.staging == 3 || (o.staging != 2 && o.precision == TF_FP64);
    shape->gap = three ? 2 : 1;
    return TF_OK;
}
// Cells per task (*B: the caller's value, or the default when it is 0) and the task shape.
tf_status task_grain(const tf_options &o, const Mesh &m, int32_t n_groups, int32_t *B, bool *patches, TaskShape *shape)
{
    tf_status s = task_shape_of(o, m, n_groups, patches, shape);
    if (s != TF_OK) return s;
    int32_t b = *B;
    if (b == 0 && *patches) {
        b = 64;  // larger patches are cut into pieces of at most 64 cells (a warp's two entry registers)
    } else if (b == 0) {
        // about 1024 units per task (at most 64 cells); 256 units and 4 to 8 cells on the
        // FP32 paired path, whose per-task cell table sets how many CTAs fit per SM (on the
        // 16^3 box with 128 directions and 16 groups, 16 cells per task left the warps waiting
        // 63 % of the sweep, 8 cells 42 % and 19 % less time)
        const bool paired = o.precision == TF_FP32 && n_groups % 2 == 0 &&
                            (o.pairing == 2 || (o.pairing == 0 && n_groups % 32 != 0));
        b = paired ? std::max(4, std::min(8, 256 / n_groups)) : std::max(2, std::min(64, 1024 / n_groups));
        // second order: a unit is a 10 x 10 solve, about 256 units per task
        if (o.order == 2) b = std::max(2, std::min(32, 256 / n_groups));
        // third order: a unit is a 20 x 20 solve, about 64 units per task (a task's time sets the
        // critical path; with the source values prefetched a pass ahead, 3 to 4 cells per task took
        // the least time on the 16^3-hex box, 128 directions, 16 groups)
        if (o.order == 3) b = std::max(1, std::min(16, 64 / n_groups));
        // trilinear hexahedra: an 8 x 8 solve, about 256 units per task and at most 8 cells when the
        // shared-matrix mode runs (G >= 8): on the paper's 16^3 grid (256 directions, 10 groups) 25
        // cells per task left the warps waiting 65 % of the sweep (3.5 ms), 8 cells 30 % (2.1 ms)
        if (m.nf == 6) b = std::max(2, std::min(n_groups >= 8 ? 8 : 32, 256 / n_groups));
        // Bulk-synchronous schedules: a bucket's tasks must cover the resident warps, and
        // most buckets hold fewer cells than the many-task grain assumes; a quarter of it
        // (at least 2 cells) took the least time over grains 1..64 on the 16^3-hex,
        // 128-direction, 16-group and the 48^3-hex, 192-direction, 64-group boxes.
        // (the quarter of the paired path's former 16-cell grain, where those measurements were made)
        if (o.schedule != TF_SCHED_AMT)
            b = std::max(2, (paired && o.order <= 1 && m.nf == 4 ? std::max(4, std::min(16, 256 / n_groups)) : b) / 4);
    }
    if (*patches && b > 64) return fail(TF_ERR_ARG, "spatial patches hold at most 64 cells");
    *B = b;
    return TF_OK;
}
}  // namespace tf

using namespace tf;

extern "C" {


void tf_options_default(tf_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = TF_FP32;
    opt->device = 0;
    opt->wait_limit_s = 10.0;
    opt->phi_accumulate = TF_PHI_PAIR;
    opt->residual_floor = 1.0;
}

const char *tf_status_string(tf_status s)
{
    switch (s) {
    case TF_OK: return "ok";
    case TF_ERR_ARG: return "invalid argument";
    case TF_ERR_MESH: return "invalid mesh";
    case TF_ERR_CYCLE: return "dependency cycle in a sweep graph";
    case TF_ERR_CUDA: return "CUDA runtime error";
    case TF_ERR_NOMEM: return "out of memory";
    case TF_ERR_TIMEOUT: return "device wait timed out";
    case TF_ERR_NOT_CONVERGED: return "not converged";
    case TF_ERR_DEVICE: return "device reported an inconsistent task graph";
    }
    return "unknown status";
}

const char *tf_last_error(void) { return g_last_error.c_str(); }

tf_status tf_mesh_create(int64_t n_vertices, const double *xyz, int64_t n_cells, const int32_t *tets, tf_handle *out)
{
    if (!out) return fail(TF_ERR_ARG, "tf_mesh_create: out is NULL");
    *out = nullptr;
    if (n_vertices < 4 || n_cells < 1 || !xyz || !tets) return fail(TF_ERR_ARG, "tf_mesh_create: empty mesh or NULL array");
    if (n_vertices >= (int64_t(1) << 31) || n_cells >= (int64_t(1) << 28))
        return fail(TF_ERR_ARG, "tf_mesh_create: at most 2^31 - 1 vertices and 2^28 - 1 cells");
    for (int64_t i = 0; i < 3 * n_vertices; ++i)
        if (!std::isfinite(xyz[i])) return fail(TF_ERR_MESH, "tf_mesh_create: non-finite coordinate");
    Mesh *m = new (std::nothrow) Mesh();
    if (!m) return fail(TF_ERR_NOMEM, "tf_mesh_create: allocation failed");
    tf_status s = build_mesh(n_vertices, xyz, n_cells, tets, *m);
    if (s != TF_OK) {
        delete m;
        return s;
    }
    *out = reinterpret_cast<tf_handle>(static_cast<Object *>(m));
    return TF_OK;
}

tf_status tf_mesh_create_hex(int64_t n_vertices, const double *xyz, int64_t n_cells, const int32_t *hexes,
                             tf_handle *out)
{
    if (!out) return fail(TF_ERR_ARG, "tf_mesh_create_hex: out is NULL");
    *out = nullptr;
    if (n_vertices < 8 || n_cells < 1 || !xyz || !hexes)
        return fail(TF_ERR_ARG, "tf_mesh_create_hex: empty mesh or NULL array");
    if (n_vertices >= (int64_t(1) << 31) || n_cells >= (int64_t(1) << 26))
        return fail(TF_ERR_ARG, "tf_mesh_create_hex: at most 2^31 - 1 vertices and 2^26 - 1 cells");
    for (int64_t i = 0; i < 3 * n_vertices; ++i)
        if (!std::isfinite(xyz[i])) return fail(TF_ERR_MESH, "tf_mesh_create_hex: non-finite coordinate");
    Mesh *m = new (std::nothrow) Mesh();
    if (!m) return fail(TF_ERR_NOMEM, "tf_mesh_create_hex: allocation failed");
    tf_status s = build_hex_mesh(n_vertices, xyz, n_cells, hexes, *m);
    if (s != TF_OK) {
        delete m;
        return s;
    }
    *out = reinterpret_cast<tf_handle>(static_cast<Object *>(m));
    return TF_OK;
}

tf_status tf_mesh_hex_integrals(tf_handle mesh, double *mass, double *grad, double *face)
{
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    if (!m || m->nf != 6) return fail(TF_ERR_ARG, "tf_mesh_hex_integrals: not a hexahedral mesh handle");
    if (mass) std::memcpy(mass, m->hmass.data(), sizeof(double) * 64 * m->nc);
    if (grad) std::memcpy(grad, m->hgrad.data(), sizeof(double) * 192 * m->nc);
    if (face) std::memcpy(face, m->hface.data(), sizeof(double) * 288 * m->nc);
    return TF_OK;
}

tf_status tf_quadrature_create(int32_t n_polar, int32_t n_azimuthal, int32_t n_dirs, const double *omega,
                               const double *w, tf_handle *out)
{
    if (!out) return fail(TF_ERR_ARG, "tf_quadrature_create: out is NULL");
    *out = nullptr;
    Quad *q = new (std::nothrow) Quad();
    if (!q) return fail(TF_ERR_NOMEM, "tf_quadrature_create: allocation failed");
    if (omega) {
        if (!w || n_dirs < 1 || n_dirs > 65535) {
            delete q;
            return fail(TF_ERR_ARG, "tf_quadrature_create: explicit set needs 1..65535 directions and weights");
        }
        q->D = n_dirs;
        q->omega.assign(omega, omega + 3 * (size_t)n_dirs);
        q->w.assign(w, w + n_dirs);
        for (int32_t a = 0; a < n_dirs; ++a) {
            const double *o = omega + 3 * a;
            const double nn = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
            if (!(std::fabs(nn - 1.0) < 1e-10) || !std::isfinite(w[a])) {
                delete q;
                return fail(TF_ERR_ARG, "tf_quadrature_create: direction " + std::to_string(a) + " is not a unit vector");
            }
        }
    } else {
        tf_status s = build_quadrature(n_polar, n_azimuthal, *q);
        if (s != TF_OK) {
            delete q;
            return s;
        }
    }
    *out = reinterpret_cast<tf_handle>(static_cast<Object *>(q));
    return TF_OK;
}

tf_status tf_problem_create(tf_handle mesh, tf_handle quad, int32_t n_groups, int32_t n_materials,
                            const int32_t *cell_material, const double *sigma_t, const double *sigma_s,
                            const double *Q, const double *S1, const double *psi_inflow, const tf_options *opt,
                            tf_handle *out)
{
    if (!out) return fail(TF_ERR_ARG, "tf_problem_create: out is NULL");
    *out = nullptr;
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    Quad *q = as<Quad>(quad, Kind::Quad);
    if (!m || !q) return fail(TF_ERR_ARG, "tf_problem_create: mesh or quadrature handle invalid");
    if (m->nf == 6 && opt && opt->order > 1)
        return fail(TF_ERR_ARG, "tf_problem_create: hexahedral meshes take the trilinear element (order 0 or 1)");
    if (n_groups < 1 || n_groups > 1024 || n_materials < 1)
        return fail(TF_ERR_ARG, "tf_problem_create: need 1 <= n_groups <= 1024 and n_materials >= 1");
    if (!cell_material || !sigma_t || !sigma_s || !Q) return fail(TF_ERR_ARG, "tf_problem_create: NULL input array");
    for (int64_t c = 0; c < m->nc; ++c)
        if (cell_material[c] < 0 || cell_material[c] >= n_materials)
            return fail(TF_ERR_ARG, "tf_problem_create: cell_material out of range at cell " + std::to_string(c));
    for (int64_t i = 0; i < (int64_t)n_materials * n_groups; ++i)
        if (!(sigma_t[i] >= 0.0) || !std::isfinite(sigma_t[i]))
            return fail(TF_ERR_ARG, "tf_problem_create: sigma_t must be finite and >= 0");
    Problem *p = new (std::nothrow) Problem();
    if (!p) return fail(TF_ERR_NOMEM, "tf_problem_create: allocation failed");
    tf_options_default(&p->opt);
    if (opt) p->opt = *opt;
    if (p->opt.precision != TF_FP32 && p->opt.precision != TF_FP64) {
        delete p;
        return fail(TF_ERR_ARG, "tf_problem_create: precision must be TF_FP32 or TF_FP64");
    }
    if (p->opt.schedule < TF_SCHED_AMT || p->opt.schedule > TF_SCHED_BSP_LAUNCH ||
        (p->opt.inject_stall && p->opt.schedule == TF_SCHED_BSP_LAUNCH)) {
        delete p;
        return fail(TF_ERR_ARG, "tf_problem_create: schedule must be a tf_schedule (inject_stall: not with "
                                "TF_SCHED_BSP_LAUNCH, which has no device wait)");
    }
    if (p->opt.order < 0 || p->opt.order > 3 ||
        (p->opt.order >= 2 && (S1 || psi_inflow))) {
        delete p;
        return fail(TF_ERR_ARG, "tf_problem_create: order must be 0 to 3 (orders 2 and 3: S1 and psi_inflow NULL)");
    }
    if (p->opt.lag_cycles != 0 && (p->opt.lag_cycles != 1 || m->nf != 6 || p->opt.task_shape == TF_TASK_PATCHES)) {
        delete p;
        return fail(TF_ERR_ARG, "tf_problem_create: lag_cycles is 0 or 1, and lagged back edges take hexahedral "
                                "meshes with t-level tasks");
    }
    if (!(p->opt.wait_limit_s > 0.0)) p->opt.wait_limit_s = 10.0;
    if (!(p->opt.residual_floor > 0.0) || p->opt.residual_floor > 1.0) p->opt.residual_floor = 1.0;
    p->mesh = m;
    p->quad = q;
    retain(m);
    retain(q);
    p->G = n_groups;
    p->M = n_materials;
    p->has_S1 = S1 != nullptr;
    p->has_inflow = psi_inflow != nullptr;
    int32_t B = p->opt.cells_per_task;
    if (B < 0 && m->nf == 6) B = 0;  // the task-grain autotuner covers tetrahedra only
    if (B < 0) {
        tf_status st = autotune_cells_per_task(*m, *q, n_groups, n_materials, cell_material, sigma_t, sigma_s, Q, p->opt,
                                               &B, &p->tune);
        if (st != TF_OK) {
            release(p);
            return st;
        }
        // the tuned kernel-variant knobs (unchanged where the caller set them)
        p->opt.pairing = p->tune.pairing;
        p->opt.staging = p->tune.staging;
        p->opt.octant_window = p->tune.window;
    }
    TaskShape shape;
    bool patches = false;
    tf_status s = task_grain(p->opt, *m, n_groups, &B, &patches, &shape);
    if (s == TF_OK) s = build_task_graph(*m, *q, B, p->graph, patches ? &shape : nullptr, p->opt.lag_cycles == 1);
    if (s == TF_OK) s = device_create(*p, cell_material, sigma_t, sigma_s, Q, S1, psi_inflow);
    if (s != TF_OK) {
        release(p);
        return s;
    }
    *out = reinterpret_cast<tf_handle>(static_cast<Object *>(p));
    return TF_OK;
}

tf_status tf_sweep(const tf_handle *problems, int32_t n, const double *const *phi_in, double *const *phi_out,
                   void *stream)
{
    if (!problems || n < 1 || !phi_in || !phi_out) return fail(TF_ERR_ARG, "tf_sweep: bad arguments");
    for (int32_t k = 0; k < n; ++k) {
        Problem *p = as<Problem>(problems[k], Kind::Problem);
        if (!p || !phi_in[k] || !phi_out[k]) return fail(TF_ERR_ARG, "tf_sweep: bad problem handle or phi pointer");
    }
    if (n > 1) return device_batch_iterate(problems, n, 0.0, 1, phi_out, nullptr, true, phi_in, stream);
    return device_sweep(*as<Problem>(problems[0], Kind::Problem), phi_in[0], phi_out[0], stream);
}

tf_status tf_source_iterate(const tf_handle *problems, int32_t n, double tol, int32_t max_iters,
                            double *const *phi, tf_iter_info *info, void *stream)
{
    if (!problems || n < 1 || !phi || max_iters < 1 || !(tol >= 0.0))
        return fail(TF_ERR_ARG, "tf_source_iterate: bad arguments");
    for (int32_t k = 0; k < n; ++k) {
        if (!as<Problem>(problems[k], Kind::Problem) || !phi[k])
            return fail(TF_ERR_ARG, "tf_source_iterate: bad problem handle or NULL phi buffer");
    }
    if (n > 1) return device_batch_iterate(problems, n, tol, max_iters, phi, info, false, nullptr, stream);
    tf_status worst = TF_OK;
    for (int32_t k = 0; k < n; ++k) {
        tf_status s = device_iterate(*as<Problem>(problems[k], Kind::Problem), tol, max_iters, phi[k],
                                     info ? info + k : nullptr, stream);
        if (s == TF_ERR_NOT_CONVERGED) {
            worst = s;
            continue;
        }
        if (s != TF_OK) return s;
    }
    return worst;
}

tf_status tf_destroy(tf_handle h)
{
    auto *o = reinterpret_cast<Object *>(h);
    if (!o) return TF_OK;
    if (o->kind != Kind::Mesh && o->kind != Kind::Quad && o->kind != Kind::Problem && o->kind != Kind::Mlp)
        return fail(TF_ERR_ARG, "tf_destroy: not a tfsweep handle");
    release(o);
    return TF_OK;
}

tf_status tf_mesh_geometry(tf_handle mesh, int64_t *n_cells, int64_t *n_vertices, double *vol, double *normal,
                           int32_t *nbr, int32_t *nbr_node)
{
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    if (!m) return fail(TF_ERR_ARG, "tf_mesh_geometry: not a mesh handle");
    if (n_cells) *n_cells = m->nc;
    if (n_vertices) *n_vertices = m->nv;
    const int64_t nf = m->nf;
    if (vol) std::memcpy(vol, m->vol.data(), sizeof(double) * m->nc);
    if (normal) std::memcpy(normal, m->normal.data(), sizeof(double) * 3 * nf * m->nc);
    if (nbr) std::memcpy(nbr, m->nbr.data(), sizeof(int32_t) * nf * m->nc);
    if (nbr_node)
        for (int64_t i = 0; i < 4 * nf * m->nc; ++i) nbr_node[i] = m->nbr_node[i];
    return TF_OK;
}

tf_status tf_quadrature_get(tf_handle quad, int32_t *n_dirs, double *omega, double *w)
{
    Quad *q = as<Quad>(quad, Kind::Quad);
    if (!q) return fail(TF_ERR_ARG, "tf_quadrature_get: not a quadrature handle");
    if (n_dirs) *n_dirs = q->D;
    if (omega) std::memcpy(omega, q->omega.data(), sizeof(double) * 3 * q->D);
    if (w) std::memcpy(w, q->w.data(), sizeof(double) * q->D);
    return TF_OK;
}

tf_status tf_graph_levels(tf_handle mesh, tf_handle quad, uint8_t *inflow, int32_t *level)
{
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    Quad *q = as<Quad>(quad, Kind::Quad);
    if (!m || !q) return fail(TF_ERR_ARG, "tf_graph_levels: mesh or quadrature handle invalid");
    return classify_and_level(*m, *q, inflow, level);
}

tf_status tf_graph_lag(tf_handle mesh, tf_handle quad, uint8_t *inflow, int32_t *level, uint8_t *lag)
{
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    Quad *q = as<Quad>(quad, Kind::Quad);
    if (!m || !q) return fail(TF_ERR_ARG, "tf_graph_lag: mesh or quadrature handle invalid");
    std::vector<uint8_t> tmp;
    if (!lag) {
        tmp.resize((size_t)q->D * m->nc);
        lag = tmp.data();
    }
    return classify_and_level(*m, *q, inflow, level, lag);
}

tf_status tf_graph_tasks(tf_handle mesh, tf_handle quad, const tf_options *opt, int32_t n_groups, int64_t *n_tasks,
                         int32_t *task_of, int32_t *position, int32_t *indeg)
{
    Mesh *m = as<Mesh>(mesh, Kind::Mesh);
    Quad *q = as<Quad>(quad, Kind::Quad);
    if (!m || !q || n_groups < 1 || n_groups > 1024) return fail(TF_ERR_ARG, "tf_graph_tasks: bad arguments");
    tf_options o;
    tf_options_default(&o);
    if (opt) o = *opt;
    if (o.cells_per_task < 0) return fail(TF_ERR_ARG, "tf_graph_tasks: the autotuned grain needs a device");
    TaskShape shape;
    bool patches = false;
    int32_t B = o.cells_per_task;
    tf_status s = task_grain(o, *m, n_groups, &B, &patches, &shape);
    if (s != TF_OK) return s;
    TaskGraph g;
    if ((s = build_task_graph(*m, *q, B, g, patches ? &shape : nullptr, o.lag_cycles == 1 && m->nf == 6 && !patches)) !=
        TF_OK)
        return s;
    if (n_tasks) *n_tasks = g.T();
    if (indeg) std::copy(g.task_indeg.begin(), g.task_indeg.end(), indeg);
    for (int64_t t = 0; t < g.T(); ++t)
        for (uint32_t i = 0; i < g.task_ncell[t]; ++i) {
            const size_t e = (size_t)g.task_cell_begin[t] + i;
            const int64_t c = g.cell_list[e] >> g.cell_shift;
            const size_t at = (size_t)g.task_dir[t] * (size_t)m->nc + (size_t)c;
            if (task_of) task_of[at] = (int32_t)t;
            if (position) position[at] = (int32_t)i;
        }
    return TF_OK;
}

tf_status tf_problem_set_reduce(tf_handle problem, tf_reduce_fn fn, void *user)
{
    Problem *p = as<Problem>(problem, Kind::Problem);
    if (!p) return fail(TF_ERR_ARG, "tf_problem_set_reduce: bad problem handle");
    p->reduce = fn;
    p->reduce_user = fn ? user : nullptr;
    return TF_OK;
}

tf_status tf_problem_psi(tf_handle problem, int32_t dir, void *out, void *stream)
{
    Problem *p = as<Problem>(problem, Kind::Problem);
    if (!p || !out) return fail(TF_ERR_ARG, "tf_problem_psi: bad handle or NULL output");
    return device_psi(*p, dir, out, stream);
}

tf_status tf_problem_stats(tf_handle problem, tf_stats *out)
{
    Problem *p = as<Problem>(problem, Kind::Problem);
    if (!p || !out) return fail(TF_ERR_ARG, "tf_problem_stats: bad handle or NULL output");
    *out = p->stats;
    out->tuned_n = p->tune.n_candidates;
    out->tuned_cached = p->tune.cached;
    out->tuned_pairing = p->tune.pairing;
    out->tuned_staging = p->tune.staging;
    out->tuned_window = p->tune.window;
    for (int k = 0; k < 8; ++k) {
        out->tuned_candidates[k] = p->tune.candidates[k];
        out->tuned_seconds[k] = p->tune.seconds[k];
    }
    return TF_OK;
}

}  // extern "C"
