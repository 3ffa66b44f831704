// Sweep graph precompute (host, once per mesh x quadrature).
//
// For every direction: classify faces (Sec. 2.1: the sweep's dependencies form
// a DAG per angle), compute t-levels (the "buckets" of the schedule), group the
// cells of one t-level into cell blocks, and derive the block-level dependency
// graph: a block's in-degree counts its distinct upwind blocks (the atomic
// counters of Sec. 3.5) and its downwind list names the blocks it releases
// (Algorithm 1's "Downwind neighbours").
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

// Levels of one direction by Kahn's algorithm; returns false on a cycle.
bool levels_one(const Mesh &m, const uint8_t *mask, int32_t *level, std::vector<int32_t> &indeg,
                std::vector<int32_t> &queue)
{
    const int64_t nc = m.nc;
    const int nf = m.nf;
    indeg.resize(nc);
    queue.resize(nc);
    int64_t tail = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int d = 0;
        for (int f = 0; f < nf; ++f) d += ((mask[c] >> f) & 1) && m.nbr[nf * c + f] >= 0;
        indeg[c] = d;
        level[c] = 0;
        if (d == 0) queue[tail++] = (int32_t)c;
    }
    for (int64_t head = 0; head < tail; ++head) {
        const int32_t c = queue[head];
        for (int f = 0; f < nf; ++f) {
            const int32_t n = m.nbr[nf * c + f];
            if (n < 0) continue;
            if (!((mask[n] >> m.nbr_face[nf * c + f]) & 1)) continue;  // n is not downwind of c
            level[n] = std::max(level[n], level[c] + 1);
            if (--indeg[n] == 0) queue[tail++] = n;
        }
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

tf_status classify_and_level(const Mesh &m, const Quad &q, uint8_t *inflow, int32_t *level)
{
    std::atomic<bool> cycle{false};
    run_parallel(q.D, [&](int32_t a) {
        std::vector<uint8_t> mask(m.nc);
        std::vector<int32_t> lev(m.nc), indeg, queue;
        for (int64_t c = 0; c < m.nc; ++c) mask[c] = inflow_mask(&q.omega[3 * a], &m.normal[3 * m.nf * c], m.nf);
        if (!levels_one(m, mask.data(), lev.data(), indeg, queue)) cycle = true;
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
    bool ok = true;
};

void build_direction(const Mesh &m, const double *O, int32_t B, DirTasks &out)
{
    const int64_t nc = m.nc;
    const int nf = m.nf, sh = nf == 6 ? 6 : 4;
    std::vector<uint8_t> mask(nc);
    std::vector<int32_t> lev(nc), indeg, queue;
    for (int64_t c = 0; c < nc; ++c) mask[c] = inflow_mask(O, &m.normal[3 * nf * c], nf);
    if (!levels_one(m, mask.data(), lev.data(), indeg, queue)) {
        out.ok = false;
        return;
    }
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
    // split every level into ceil(m / B) blocks of balanced size
    std::vector<int32_t> block_of(nc);
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
                if (((mask[c] >> f) & 1) && m.nbr[nf * c + f] >= 0) tmp.push_back(block_of[m.nbr[nf * c + f]]);
        }
        std::sort(tmp.begin(), tmp.end());
        out.indeg[b] = (int32_t)(std::unique(tmp.begin(), tmp.end()) - tmp.begin());
        // downwind blocks: neighbours whose matching face is inflow
        tmp.clear();
        for (uint32_t i = out.cell_begin[b]; i < out.cell_begin[b] + out.ncell[b]; ++i) {
            const int32_t c = (int32_t)(out.cells[i] >> sh);
            for (int f = 0; f < nf; ++f) {
                const int32_t n = m.nbr[nf * c + f];
                if (n >= 0 && ((mask[n] >> m.nbr_face[nf * c + f]) & 1)) tmp.push_back(block_of[n]);
            }
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        out.down.insert(out.down.end(), tmp.begin(), tmp.end());
        out.down_begin[b + 1] = (uint32_t)out.down.size();
    }
    // b-level: longest chain of downwind blocks below each block (blocks are in level order)
    out.blevel.assign(T, 0);
    for (int32_t b = T - 1; b >= 0; --b) {
        int32_t v = 0;
        for (uint32_t k = out.down_begin[b]; k < out.down_begin[b + 1]; ++k) v = std::max(v, 1 + out.blevel[out.down[k]]);
        out.blevel[b] = v;
    }
}

}  // namespace

tf_status build_task_graph(const Mesh &m, const Quad &q, int32_t B, TaskGraph &g)
{
    if (B < 1 || B > 4096) return fail(TF_ERR_ARG, "cells_per_task must be in [1, 4096]");
    const int sh = m.nf == 6 ? 6 : 4;
    if (m.nc >= (int64_t(1) << (32 - sh)))
        return fail(TF_ERR_ARG, "mesh too large: at most 2^" + std::to_string(32 - sh) + " - 1 cells");
    std::vector<DirTasks> per(q.D);
    try {
        run_parallel(q.D, [&](int32_t a) { build_direction(m, &q.omega[3 * a], B, per[a]); });
    } catch (const std::bad_alloc &) {
        return fail(TF_ERR_NOMEM, "graph: host allocation failed");
    }
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
    return TF_OK;
}

}  // namespace tf
