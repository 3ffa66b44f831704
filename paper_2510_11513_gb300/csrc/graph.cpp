// Sweep graph precompute (host, once per mesh x quadrature).
//
// For every direction: classify faces (Sec. 2.1: the sweep's dependencies form
// a DAG per angle), compute t-levels (the "buckets" of the schedule), group the
// cells into tasks, and derive the task-level dependency graph: a task's
// in-degree counts its distinct upwind tasks (the atomic counters of Sec. 3.5)
// and its downwind list names the tasks it releases (Algorithm 1's "Downwind
// neighbours").  Two task shapes (the granularity question of Sec. 3.4):
//   - t-level blocks: up to B cells of one t-level (independent of each other);
//   - spatial patches: cells of one small box of space, in an order that respects
//     their dependencies, so that most upwind face traces a task's cells need are
//     produced inside the same task and never leave the chip.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <thread>

#include "tf_internal.h"

namespace tf {

namespace {

// inflow iff Omega . N_f < -1e-12 |N_f|, dot product as ((Ox Nx + Oy Ny) + Oz Nz)
inline uint8_t inflow_mask(const double *O, const double *Nc, int nf)
{
    uint8_t m = 0;
    for (int f = 0; f < nf; ++f) {
        const double *N = Nc + 3 * f;
        const double s = (O[0] * N[0] + O[1] * N[1]) + O[2] * N[2];
        const double eps = 1e-12 * std::sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
        if (s < -eps) m |= (uint8_t)(1u << f);
    }
    return m;
}

// Levels of one direction by Kahn's algorithm; returns false on a cycle.  With lag
// (non-null, [nc]) cycles are broken instead: whenever no cell is ready, a walk from
// the lowest-numbered waiting cell steps to the upwind neighbour across its
// lowest-numbered open face (inflow, interior, not reached, not lagged) until it comes
// back to a cell it has visited; the face it would cross then closes a cycle and is
// lagged (lag[c] bit f: the kernel reads the previous transport step's upwind values
// there), and the ordering continues.  Lagged faces do not count for the levels.
bool levels_one(const Mesh &m, const uint8_t *mask, int32_t *level, std::vector<int32_t> &indeg,
                std::vector<int32_t> &queue, uint8_t *lag = nullptr)
{
    const int64_t nc = m.nc;
    const int nf = m.nf;
    indeg.resize(nc);
    queue.resize(nc);
    std::vector<uint8_t> reached(nc);
    std::vector<int64_t> walk(lag ? nc : 0, -1);
    int64_t tail = 0, head = 0, next = 0, stamp = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int d = 0;
        for (int f = 0; f < nf; ++f) d += ((mask[c] >> f) & 1) && m.nbr[nf * c + f] >= 0;
        indeg[c] = d;
        level[c] = 0;
        reached[c] = d == 0;
        if (lag) lag[c] = 0;
        if (d == 0) queue[tail++] = (int32_t)c;
    }
    for (;;) {
        for (; head < tail; ++head) {
            const int32_t c = queue[head];
            for (int f = 0; f < nf; ++f) {
                const int32_t n = m.nbr[nf * c + f];
                if (n < 0 || reached[n]) continue;
                const int fn = m.nbr_face[nf * c + f];
                if (!((mask[n] >> fn) & 1)) continue;        // n is not downwind of c
                if (lag && ((lag[n] >> fn) & 1)) continue;   // lagged: not a dependency
                level[n] = std::max(level[n], level[c] + 1);
                if (--indeg[n] == 0) {
                    reached[n] = 1;
                    queue[tail++] = n;
                }
            }
        }
        if (tail == nc || !lag) break;
        while (reached[next]) ++next;
        int64_t cur = next;
        walk[cur] = stamp;
        for (;;) {
            int fo = -1;
            int32_t n = -1;
            for (int f = 0; f < nf && fo < 0; ++f) {
                n = m.nbr[nf * cur + f];
                if (((mask[cur] >> f) & 1) && !((lag[cur] >> f) & 1) && n >= 0 && !reached[n]) fo = f;
            }
            if (fo < 0) return false;  // a waiting cell always waits on someone; never taken
            if (walk[n] == stamp) {    // cur -> n closes a cycle: lag that face
                lag[cur] |= (uint8_t)(1u << fo);
                if (--indeg[cur] == 0) {
                    reached[cur] = 1;
                    queue[tail++] = (int32_t)cur;
                }
                break;
            }
            walk[n] = stamp;
            cur = n;
        }
        ++stamp;
    }
    return tail == nc;
}

void run_parallel(int32_t D, const std::function<void(int32_t)> &fn)
{
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
    nt = std::min<unsigned>(nt, (unsigned)std::max(1, D));
    std::atomic<int32_t> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (int32_t a; (a = next.fetch_add(1)) < D;) fn(a);
        });
    for (auto &t : th) t.join();
}

}  // namespace

tf_status classify_and_level(const Mesh &m, const Quad &q, uint8_t *inflow, int32_t *level, uint8_t *lag)
{
    std::atomic<bool> cycle{false};
    run_parallel(q.D, [&](int32_t a) {
        std::vector<uint8_t> mask(m.nc);
        std::vector<int32_t> lev(m.nc), indeg, queue;
        for (int64_t c = 0; c < m.nc; ++c) mask[c] = inflow_mask(&q.omega[3 * a], &m.normal[3 * m.nf * c], m.nf);
        if (!levels_one(m, mask.data(), lev.data(), indeg, queue, lag ? lag + (size_t)a * m.nc : nullptr))
            cycle = true;
        if (inflow) std::copy(mask.begin(), mask.end(), inflow + (size_t)a * m.nc);
        if (level) std::copy(lev.begin(), lev.end(), level + (size_t)a * m.nc);
    });
    if (cycle) return fail(TF_ERR_CYCLE, "graph: a direction's dependency graph has a cycle");
    return TF_OK;
}

namespace {

struct DirTasks {
    int32_t levels = 0;
    std::vector<uint32_t> cells;       // (cell << shift) | mask, in task order
    std::vector<uint32_t> cell_begin;  // per task, local into cells
    std::vector<uint16_t> ncell;
    std::vector<int32_t> level;
    std::vector<int32_t> indeg;
    std::vector<int32_t> blevel;
    std::vector<uint32_t> down_begin;  // per task + 1
    std::vector<uint32_t> down;        // local task ids
    std::vector<uint8_t> lag;          // lagged faces of each cell entry, in task order (empty: none)
    bool ok = true;
};

// Spatial patches of one direction.  Every cell gets a round: 0 without interior
// inflow faces, else the largest over its upwind cells u of round(u), plus one
// when u lies in another region.  The cells of one (round, region) pair form a
// patch (split into pieces of at most B cells).  Every edge between two patches
// then goes from a lower round to a higher one, or between pieces of one patch in
// their order, so the patch graph has no cycle, whatever the regions look like.
// Inside a patch the cells are listed in an order that respects their
// dependencies; a cell that depends on one of the `gap` cells listed just
// before it is avoided when another is ready (the kernel stages a cell's inputs
// `gap` cells ahead, and such a trace cannot be staged from memory).
void patch_tasks(const Mesh &m, const uint8_t *mask, const int32_t *lev, const std::vector<int32_t> &order,
                 const std::vector<int32_t> &region, int32_t B, int32_t gap, std::vector<int32_t> &task_of,
                 DirTasks &out)
{
    const int64_t nc = m.nc;
    const int nf = m.nf, sh = nf == 6 ? 6 : 4;
    auto upwind = [&](int64_t c, int f) -> int32_t {
        const int32_t n = m.nbr[nf * c + f];
        return (((mask[c] >> f) & 1) && n >= 0) ? n : -1;
    };
    std::vector<int32_t> rnd(nc, 0);
    for (int64_t i = 0; i < nc; ++i) {  // t-level order is a topological order
        const int32_t c = order[i];
        int32_t r = 0;
        for (int f = 0; f < nf; ++f) {
            const int32_t u = upwind(c, f);
            if (u >= 0) r = std::max(r, rnd[u] + (region[u] != region[c] ? 1 : 0));
        }
        rnd[c] = r;
    }
    // cells grouped by (round, region), t-level order inside a group (stable sort of the level order)
    std::vector<int32_t> by(order);
    std::stable_sort(by.begin(), by.end(), [&](int32_t x, int32_t y) {
        return rnd[x] != rnd[y] ? rnd[x] < rnd[y] : region[x] < region[y];
    });
    out.cells.resize(nc);
    std::vector<int32_t> pos_in(nc, -1), indeg_in, picked;
    std::vector<uint8_t> done;
    int64_t w = 0;
    for (int64_t g0 = 0; g0 < nc;) {
        int64_t g1 = g0 + 1;
        while (g1 < nc && rnd[by[g1]] == rnd[by[g0]] && region[by[g1]] == region[by[g0]]) ++g1;
        const int64_t n = g1 - g0;
        for (int64_t k = 0; k < n; ++k) pos_in[by[g0 + k]] = (int32_t)k;
        indeg_in.assign(n, 0);
        done.assign(n, 0);
        for (int64_t k = 0; k < n; ++k)
            for (int f = 0; f < nf; ++f) {
                const int32_t u = upwind(by[g0 + k], f);
                if (u >= 0 && pos_in[u] >= 0) ++indeg_in[k];
            }
        // list scheduling: the first ready cell in t-level order that does not depend on the
        // last `gap` listed cells, else the first ready cell
        picked.clear();
        for (int64_t step = 0; step < n; ++step) {
            int64_t pick = -1, first = -1;
            for (int64_t k = 0; k < n && pick < 0; ++k) {
                if (done[k] || indeg_in[k] != 0) continue;
                if (first < 0) first = k;
                bool near = false;
                for (int f = 0; f < nf && !near; ++f) {
                    const int32_t u = upwind(by[g0 + k], f);
                    if (u < 0 || pos_in[u] < 0) continue;
                    for (int64_t j = (int64_t)picked.size() - 1; j >= 0 && j >= (int64_t)picked.size() - gap; --j)
                        if (picked[j] == pos_in[u]) near = true;
                }
                if (!near) pick = k;
            }
            if (pick < 0) pick = first;
            done[pick] = 1;
            picked.push_back((int32_t)pick);
            const int32_t c = by[g0 + pick];
            for (int f = 0; f < nf; ++f) {  // downwind cells of c inside the group
                const int32_t d = m.nbr[nf * c + f];
                if (d >= 0 && pos_in[d] >= 0 && ((mask[d] >> m.nbr_face[nf * c + f]) & 1)) --indeg_in[pos_in[d]];
            }
        }
        // pieces of at most B cells, in the listed order
        const int64_t np = (n + B - 1) / B;
        for (int64_t k = 0; k < np; ++k) {
            const int64_t s = (n * k) / np, e = (n * (k + 1)) / np;
            const int32_t id = (int32_t)out.ncell.size();
            out.cell_begin.push_back((uint32_t)(w));
            out.ncell.push_back((uint16_t)(e - s));
            out.level.push_back(rnd[by[g0]]);
            for (int64_t i = s; i < e; ++i) {
                const int32_t c = by[g0 + picked[i]];
                task_of[c] = id;
                out.cells[w++] = ((uint32_t)c << sh) | mask[c];
            }
        }
        for (int64_t k = 0; k < n; ++k) pos_in[by[g0 + k]] = -1;
        g0 = g1;
    }
}

void build_direction(const Mesh &m, const double *O, int32_t B, const std::vector<int32_t> *region, int32_t gap,
                     bool lag_cycles, DirTasks &out)
{
    const int64_t nc = m.nc;
    const int nf = m.nf, sh = nf == 6 ? 6 : 4;
    std::vector<uint8_t> mask(nc), lagc(lag_cycles ? nc : 0);
    std::vector<int32_t> lev(nc), indeg, queue;
    for (int64_t c = 0; c < nc; ++c) mask[c] = inflow_mask(O, &m.normal[3 * nf * c], nf);
    if (!levels_one(m, mask.data(), lev.data(), indeg, queue, lag_cycles ? lagc.data() : nullptr)) {
        out.ok = false;
        return;
    }
    bool any_lag = false;
    for (uint8_t v : lagc) any_lag |= v != 0;
    // a lagged face is not a dependency
    auto dep = [&](int64_t c, int f) { return ((mask[c] >> f) & 1) && !(any_lag && ((lagc[c] >> f) & 1)); };
    int32_t L = 0;
    for (int64_t c = 0; c < nc; ++c) L = std::max(L, lev[c] + 1);
    out.levels = L;
    // cells ordered by (level, cell id)
    std::vector<int64_t> lstart(L + 1, 0);
    for (int64_t c = 0; c < nc; ++c) lstart[lev[c] + 1]++;
    for (int32_t l = 0; l < L; ++l) lstart[l + 1] += lstart[l];
    std::vector<int32_t> order(nc);
    {
        std::vector<int64_t> pos(lstart.begin(), lstart.end() - 1);
        for (int64_t c = 0; c < nc; ++c) order[pos[lev[c]]++] = (int32_t)c;
    }
    std::vector<int32_t> block_of(nc);
    if (region) {
        patch_tasks(m, mask.data(), lev.data(), order, *region, B, gap, block_of, out);
    } else {
        // split every level into ceil(m / B) blocks of balanced size
        out.cells.resize(nc);
        for (int32_t l = 0; l < L; ++l) {
            const int64_t b0 = lstart[l], mcount = lstart[l + 1] - lstart[l];
            const int64_t nb = (mcount + B - 1) / B;
            for (int64_t k = 0; k < nb; ++k) {
                const int64_t s = b0 + (mcount * k) / nb, e = b0 + (mcount * (k + 1)) / nb;
                const int32_t id = (int32_t)out.ncell.size();
                out.cell_begin.push_back((uint32_t)s);
                out.ncell.push_back((uint16_t)(e - s));
                out.level.push_back(l);
                for (int64_t i = s; i < e; ++i) {
                    const int32_t c = order[i];
                    block_of[c] = id;
                    out.cells[i] = ((uint32_t)c << sh) | mask[c];
                }
            }
        }
    }
    const int32_t T = (int32_t)out.ncell.size();
    out.indeg.assign(T, 0);
    out.down_begin.assign(T + 1, 0);
    std::vector<int32_t> tmp;
    for (int32_t b = 0; b < T; ++b) {
        // upwind blocks: neighbours across interior inflow faces
        tmp.clear();
        for (uint32_t i = out.cell_begin[b]; i < out.cell_begin[b] + out.ncell[b]; ++i) {
            const int32_t c = (int32_t)(out.cells[i] >> sh);
            for (int f = 0; f < nf; ++f)
                if (dep(c, f) && m.nbr[nf * c + f] >= 0 && block_of[m.nbr[nf * c + f]] != b)
                    tmp.push_back(block_of[m.nbr[nf * c + f]]);
        }
        std::sort(tmp.begin(), tmp.end());
        out.indeg[b] = (int32_t)(std::unique(tmp.begin(), tmp.end()) - tmp.begin());
        // downwind blocks: neighbours whose matching face is inflow
        tmp.clear();
        for (uint32_t i = out.cell_begin[b]; i < out.cell_begin[b] + out.ncell[b]; ++i) {
            const int32_t c = (int32_t)(out.cells[i] >> sh);
            for (int f = 0; f < nf; ++f) {
                const int32_t n = m.nbr[nf * c + f];
                if (n >= 0 && dep(n, m.nbr_face[nf * c + f]) && block_of[n] != b) tmp.push_back(block_of[n]);
            }
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        out.down.insert(out.down.end(), tmp.begin(), tmp.end());
        out.down_begin[b + 1] = (uint32_t)out.down.size();
    }
    if (any_lag) {
        out.lag.resize(out.cells.size());
        for (size_t i = 0; i < out.cells.size(); ++i) out.lag[i] = lagc[out.cells[i] >> sh];
    }
    // b-level: longest chain of downwind tasks below each task (tasks are in a topological
    // order: t-level blocks by level, patches by round and, inside a patch, by piece)
    out.blevel.assign(T, 0);
    for (int32_t b = T - 1; b >= 0; --b) {
        int32_t v = 0;
        for (uint32_t k = out.down_begin[b]; k < out.down_begin[b + 1]; ++k) v = std::max(v, 1 + out.blevel[out.down[k]]);
        out.blevel[b] = v;
    }
}

}  // namespace

// Regions of the spatial patches: boxes of edge `extent` times the mean cell size
// (the edge of a cube holding six tetrahedra of the mean volume, or one hexahedron),
// aligned with the mesh's bounding box; a cell belongs to the box holding its
// vertex centroid.
static void patch_regions(const Mesh &m, double extent, std::vector<int32_t> &region)
{
    const int nv_cell = m.nf == 6 ? 8 : 4;
    const int32_t *cv = m.nf == 6 ? m.hexes.data() : m.tets.data();
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, vol = 0.0;
    for (int64_t v = 0; v < m.nv; ++v)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], m.xyz[3 * v + d]);
            hi[d] = std::max(hi[d], m.xyz[3 * v + d]);
        }
    for (int64_t c = 0; c < m.nc; ++c) vol += m.vol[c];
    const double h = std::cbrt((m.nf == 6 ? 1.0 : 6.0) * vol / (double)std::max<int64_t>(1, m.nc));
    const double edge = std::max(extent, 1e-3) * h;
    int64_t nb[3];
    for (int d = 0; d < 3; ++d) nb[d] = std::max<int64_t>(1, (int64_t)std::floor((hi[d] - lo[d]) / edge) + 1);
    region.resize(m.nc);
    for (int64_t c = 0; c < m.nc; ++c) {
        int64_t b[3];
        for (int d = 0; d < 3; ++d) {
            double x = 0.0;
            for (int k = 0; k < nv_cell; ++k) x += m.xyz[3 * (int64_t)cv[nv_cell * c + k] + d];
            x /= nv_cell;
            b[d] = std::min(nb[d] - 1, std::max<int64_t>(0, (int64_t)std::floor((x - lo[d]) / edge)));
        }
        region[c] = (int32_t)((b[0] + nb[0] * (b[1] + nb[1] * b[2])) % 2147483647);
    }
}

tf_status build_task_graph(const Mesh &m, const Quad &q, int32_t B, TaskGraph &g, const TaskShape *shape,
                           bool lag_cycles)
{
    if (lag_cycles && shape) return fail(TF_ERR_ARG, "lagged back edges take t-level tasks, not spatial patches");
    if (B < 1 || B > 4096) return fail(TF_ERR_ARG, "cells_per_task must be in [1, 4096]");
    const int sh = m.nf == 6 ? 6 : 4;
    if (m.nc >= (int64_t(1) << (32 - sh)))
        return fail(TF_ERR_ARG, "mesh too large: at most 2^" + std::to_string(32 - sh) + " - 1 cells");
    if (shape && (B > 64 || shape->gap < 0 || shape->gap > 8))
        return fail(TF_ERR_ARG, "spatial patches: at most 64 cells per task");
    std::vector<DirTasks> per(q.D);
    std::vector<int32_t> region;
    try {
        if (shape) patch_regions(m, shape->extent, region);
        run_parallel(q.D, [&](int32_t a) {
            build_direction(m, &q.omega[3 * a], B, shape ? &region : nullptr, shape ? shape->gap : 0, lag_cycles,
                            per[a]);
        });
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "graph: host allocation failed");
    }
    g.patches = shape != nullptr;
    for (auto &d : per)
        if (!d.ok) return fail(TF_ERR_CYCLE, "graph: a direction's dependency graph has a cycle");
    g.D = q.D;
    g.cells_per_task = B;
    g.cell_shift = sh;
    g.dir_task_begin.assign(q.D + 1, 0);
    g.dir_levels.resize(q.D);
    int64_t T = 0, E = 0;
    g.max_level = 0;
    for (int32_t a = 0; a < q.D; ++a) {
        g.dir_task_begin[a] = T;
        T += (int64_t)per[a].ncell.size();
        E += (int64_t)per[a].down.size();
        g.dir_levels[a] = per[a].levels;
        g.max_level = std::max(g.max_level, per[a].levels - 1);
    }
    g.dir_task_begin[q.D] = T;
    if (T >= (int64_t(1) << 32) || (int64_t)q.D * m.nc >= (int64_t(1) << 32))
        return fail(TF_ERR_ARG, "graph: more than 2^32 tasks or cell entries");
    try {
        g.task_cell_begin.resize(T);
        g.task_ncell.resize(T);
        g.task_dir.resize(T);
        g.task_level.resize(T);
        g.task_indeg.resize(T);
        g.task_blevel.resize(T);
        g.down_begin.resize(T + 1);
        g.down_list.resize(E);
        g.cell_list.resize((size_t)q.D * m.nc);
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "graph: host allocation failed");
    }
    std::vector<int64_t> ebeg(q.D + 1, 0);
    for (int32_t a = 0; a < q.D; ++a) ebeg[a + 1] = ebeg[a] + (int64_t)per[a].down.size();
    run_parallel(q.D, [&](int32_t a) {
        const DirTasks &d = per[a];
        const int64_t t0 = g.dir_task_begin[a];
        const uint64_t cell0 = (uint64_t)a * m.nc;
        std::copy(d.cells.begin(), d.cells.end(), g.cell_list.begin() + cell0);
        for (size_t b = 0; b < d.ncell.size(); ++b) {
            g.task_cell_begin[t0 + b] = (uint32_t)(cell0 + d.cell_begin[b]);
            g.task_ncell[t0 + b] = d.ncell[b];
            g.task_dir[t0 + b] = (uint16_t)a;
            g.task_level[t0 + b] = d.level[b];
            g.task_indeg[t0 + b] = d.indeg[b];
            g.task_blevel[t0 + b] = d.blevel[b];
            g.down_begin[t0 + b] = (uint64_t)ebeg[a] + d.down_begin[b];
        }
        for (size_t k = 0; k < d.down.size(); ++k) g.down_list[ebeg[a] + k] = (uint32_t)(t0 + d.down[k]);
    });
    g.down_begin[T] = (uint64_t)E;
    // lagged back edges: per cell entry (lag mask << 26) | first slot, slots numbered by
    // direction, entry and face; per slot its direction and (cell << 3) | face
    g.cell_lag.clear();
    g.lag_slots.clear();
    g.lag_dir_begin.assign(q.D + 1, 0);
    bool any = false;
    for (auto &d : per) any |= !d.lag.empty();
    if (any) {
        g.cell_lag.assign(g.cell_list.size(), 0u);
        int64_t slot = 0;
        for (int32_t a = 0; a < q.D; ++a) {
            g.lag_dir_begin[a] = slot;
            const DirTasks &d = per[a];
            for (size_t i = 0; i < d.lag.size(); ++i) {
                if (!d.lag[i]) continue;
                if (slot >= (int64_t(1) << 26)) return fail(TF_ERR_ARG, "graph: more than 2^26 lagged faces");
                const uint64_t pos = (uint64_t)a * m.nc + i;
                g.cell_lag[pos] = ((uint32_t)d.lag[i] << 26) | (uint32_t)slot;
                const uint32_t c = d.cells[i] >> sh;
                for (int f = 0; f < m.nf; ++f)
                    if ((d.lag[i] >> f) & 1) {
                        g.lag_slots.push_back((uint32_t)a);
                        g.lag_slots.push_back((c << 3) | (uint32_t)f);
                        ++slot;
                    }
            }
        }
        g.lag_dir_begin[q.D] = slot;
    }
    return TF_OK;
}

}  // namespace tf
