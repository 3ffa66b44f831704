// Autotuner: picks a problem's task grain (cells_per_task), then its kernel
// variant (groups per lane: packed group pairs or one group; shared-memory staging
// or registers) and the octant window (how many octants' directions are in the
// ready queue at once), by timing trial sweeps of the same mesh, groups and cross
// sections over a sample of its directions.  Only knobs the caller left automatic
// are tuned.  The choice is cached per (precision, order, schedule, criterion,
// groups, directions, log2 cells).  Criterion: the wall time of the trial sweep
// (cells_per_task = -1, a problem swept on its own) or the summed busy time of the
// warps (-2, a problem swept in a batch, where the other problems keep the GPU busy).
// The direction chunk is not tuned: the fewest chunks the memory allows is always
// fastest (each chunk repeats the fill, the launch tail and the phi pass).  The default
// choice is the incumbent; a candidate replaces it only when at least 5 % faster.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "tf_internal.h"

namespace tf {

namespace {

struct Choice {
    int32_t cells = 0, pairing = 0, staging = 0, window = 0;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, Choice> g_cache;

}  // namespace

tf_status autotune_cells_per_task(const Mesh &m, const Quad &q, int32_t G, int32_t M, const int32_t *cell_material,
                                  const double *sigma_t, const double *sigma_s, const double *Q, const tf_options &opt,
                                  int32_t *out, tf_autotune_report *rep)
{
    const int lc = (int)std::lround(std::log2((double)std::max<int64_t>(m.nc, 1)));
    const auto key = std::make_tuple(opt.task_shape * 256 + opt.precision * 64 + opt.order * 16 + opt.schedule * 4 +
                                         (opt.cells_per_task == -2 ? 1 : 0),
                                     G, q.D, lc);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *out = it->second.cells;
            if (rep) {
                rep->cached = 1;
                rep->pairing = it->second.pairing;
                rep->staging = it->second.staging;
                rep->window = it->second.window;
            }
            return TF_OK;
        }
    }
    // direction sample: up to 32 directions spread over the set
    const int Ds = std::min(q.D, 32);
    Quad *qs = new Quad();
    qs->D = Ds;
    for (int k = 0; k < Ds; ++k) {
        const int a = (int)((int64_t)k * q.D / Ds);
        qs->omega.insert(qs->omega.end(), &q.omega[3 * a], &q.omega[3 * a] + 3);
        qs->w.push_back(q.w[a]);
    }
    const bool fp32 = opt.precision == TF_FP32, order1 = opt.order != 2;
    const bool paired = order1 && fp32 && G % 2 == 0 && (opt.pairing == 2 || (opt.pairing == 0 && G % 32 != 0));
    const int cap = (!order1 || paired) ? 32 : 64;
    // the default grain is the incumbent: another candidate replaces it only when its trial is
    // at least 5 % faster (trial sweeps over a direction sample are noisy at that level)
    int32_t b_def = 0;
    {
        tf_options o = opt;
        o.cells_per_task = 0;
        bool pt = false;
        TaskShape sh;
        if (task_grain(o, m, G, &b_def, &pt, &sh) != TF_OK) b_def = std::max(2, std::min(cap, 1024 / G));
    }
    std::vector<int32_t> cand{b_def};
    for (int32_t b : {2, 4, 8, 16, 32, 64})
        if (b != b_def && (b > 2 || opt.schedule != TF_SCHED_AMT) && b <= cap && (int64_t)b * G <= 4096)
            cand.push_back(b);
    const int nb = order1 ? 4 : (opt.order == 3 ? 20 : 10);
    std::vector<double> phi((size_t)m.nc * G * nb, 1.0);
    double *dphi = nullptr;
    if (cudaMalloc(&dphi, phi.size() * 8) != cudaSuccess) {
        delete qs;
        return fail(TF_ERR_NOMEM, "autotune: device allocation failed");
    }
    cudaMemcpy(dphi, phi.data(), phi.size() * 8, cudaMemcpyHostToDevice);
    // One trial: the problem on the direction sample, one warm-up sweep, the best of two
    // timed sweeps.  On its own the wall time counts; in a batch (other problems supply
    // the parallelism) the warps' busy time, i.e. the cost of the units on a saturated GPU.
    auto trial = [&](const tf_options &o) -> double {
        Problem *p = new Problem();
        p->opt = o;
        p->opt.dir_chunk = 0;
        p->opt.psi_budget_gb = 0;
        p->mesh = const_cast<Mesh *>(&m);
        p->quad = qs;
        retain(p->mesh);
        retain(p->quad);
        p->G = G;
        p->M = M;
        TaskShape shape;
        bool patches = false;
        tf_status s = task_shape_of(o, m, G, &patches, &shape);
        if (s == TF_OK) s = build_task_graph(m, *qs, o.cells_per_task, p->graph, patches ? &shape : nullptr);
        if (s == TF_OK) s = device_create(*p, cell_material, sigma_t, sigma_s, Q, nullptr, nullptr);
        double t = 1e300;
        if (s == TF_OK) {
            s = device_sweep(*p, dphi, dphi, nullptr);
            for (int r = 0; r < 2 && s == TF_OK; ++r) {
                cudaDeviceSynchronize();
                const auto t0 = std::chrono::steady_clock::now();
                s = device_sweep(*p, dphi, dphi, nullptr);
                const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                t = std::min(t, opt.cells_per_task == -2 ? p->stats.busy_seconds : wall);
            }
        }
        release(p);
        return s == TF_OK ? t : -1.0;
    };
    // phase 1: the grain, with the variant knobs as the caller gave them
    double best_t = 1e300;
    Choice best{cand[0], opt.pairing, opt.staging, opt.octant_window};
    int tried = 0;
    for (int32_t b : cand) {
        tf_options o = opt;
        o.cells_per_task = b;
        const double t = trial(o);
        if (rep && tried < 8) {
            rep->candidates[tried] = b;
            rep->seconds[tried] = t;
        }
        ++tried;
        if (t >= 0.0 && t < (b == b_def ? best_t : 0.95 * best_t)) {
            best_t = t;
            best.cells = b;
        }
    }
    // phase 2: at that grain, the other group-per-lane variant, registers instead of
    // shared-memory staging, and two octants in the ready queue instead of all
    std::vector<Choice> vars;
    if (opt.pairing == 0 && order1 && fp32 && G % 2 == 0 && best.cells <= 32)
        vars.push_back({best.cells, G % 32 == 0 ? 2 : 1, best.staging, best.window});
    if (opt.staging == 0 && G % 32 == 0 && (order1 || (fp32 && opt.order == 2)))
        vars.push_back({best.cells, best.pairing, 1, best.window});
    if (opt.octant_window == 0 && opt.schedule == TF_SCHED_AMT) vars.push_back({best.cells, best.pairing, best.staging, 2});
    int nvar = 0;
    for (const Choice &v : vars) {
        tf_options o = opt;
        o.cells_per_task = v.cells;
        o.pairing = v.pairing;
        o.staging = v.staging;
        o.octant_window = v.window;
        const double t = trial(o);
        ++nvar;
        if (t >= 0.0 && t < 0.95 * best_t) {
            best_t = t;
            best = v;
        }
    }
    cudaFree(dphi);
    release(qs);
    if (rep) {
        rep->n_candidates = std::min(tried, 8);
        rep->chosen = best.cells;
        rep->cached = 0;
        rep->sample_directions = Ds;
        rep->pairing = best.pairing;
        rep->staging = best.staging;
        rep->window = best.window;
        rep->n_variants = nvar;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = best;
    }
    *out = best.cells;
    return TF_OK;
}

}  // namespace tf
