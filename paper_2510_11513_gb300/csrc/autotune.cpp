// Task-grain autotuner: picks cells_per_task for a problem by timing trial
// sweeps of the same mesh, groups and cross sections over a sample of its
// directions, one candidate grain at a time; the choice is cached per
// (precision, criterion, groups, directions, log2 cells).  Criterion: the wall
// time of the trial sweep (cells_per_task = -1, a problem swept on its own) or
// the summed busy time of the warps (-2, a problem swept in a batch, where the
// other problems keep the GPU busy).  The trial sweeps use the problem's own
// schedule (many-task or bulk-synchronous), which is part of the cache key.
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

std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, int32_t> g_cache;

}  // namespace

tf_status autotune_cells_per_task(const Mesh &m, const Quad &q, int32_t G, int32_t M, const int32_t *cell_material,
                                  const double *sigma_t, const double *sigma_s, const double *Q, const tf_options &opt,
                                  int32_t *out, tf_autotune_report *rep)
{
    const int lc = (int)std::lround(std::log2((double)std::max<int64_t>(m.nc, 1)));
    const auto key =
        std::make_tuple(opt.precision * 16 + opt.schedule * 4 + (opt.cells_per_task == -2 ? 1 : 0), G, q.D, lc);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *out = it->second;
            if (rep) rep->cached = 1;
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
    const bool paired = opt.precision == TF_FP32 && G % 2 == 0 && (opt.pairing == 2 || (opt.pairing == 0 && G % 32 != 0));
    const int cap = paired ? 32 : 64;
    std::vector<int32_t> cand;
    for (int32_t b : {2, 4, 8, 16, 32, 64})
        if ((b > 2 || opt.schedule != TF_SCHED_AMT) && b <= cap && (int64_t)b * G <= 4096) cand.push_back(b);
    if (cand.empty()) cand.push_back(std::max(2, std::min(cap, 1024 / G)));
    std::vector<double> phi((size_t)m.nc * G * 4, 0.0);
    for (size_t i = 0; i < phi.size(); ++i) phi[i] = 1.0;
    double *dphi = nullptr;
    if (cudaMalloc(&dphi, phi.size() * 8) != cudaSuccess) {
        delete qs;
        return fail(TF_ERR_NOMEM, "autotune: device allocation failed");
    }
    cudaMemcpy(dphi, phi.data(), phi.size() * 8, cudaMemcpyHostToDevice);
    double best_t = 1e300;
    int32_t best = cand[0];
    int tried = 0;
    for (int32_t b : cand) {
        tf_options o = opt;
        o.cells_per_task = b;
        o.dir_chunk = 0;
        o.psi_budget_gb = 0;
        Problem *p = new Problem();
        p->opt = o;
        p->mesh = const_cast<Mesh *>(&m);
        p->quad = qs;
        retain(p->mesh);
        retain(p->quad);
        p->G = G;
        p->M = M;
        tf_status s = build_task_graph(m, *qs, b, p->graph);
        if (s == TF_OK) s = device_create(*p, cell_material, sigma_t, sigma_s, Q, nullptr, nullptr);
        double t = 1e300;
        if (s == TF_OK) {
            // one warm-up sweep, then the best of two timed sweeps.  For use on its own the
            // wall time counts; for batched use (other problems supply the parallelism) the
            // warps' busy time, i.e. the cost of the units when the GPU is saturated.
            s = device_sweep(*p, dphi, dphi, nullptr);
            for (int r = 0; r < 2 && s == TF_OK; ++r) {
                cudaDeviceSynchronize();
                const auto t0 = std::chrono::steady_clock::now();
                s = device_sweep(*p, dphi, dphi, nullptr);
                const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                t = std::min(t, opt.cells_per_task == -2 ? p->stats.busy_seconds : wall);
            }
        }
        if (rep && tried < 8) {
            rep->candidates[tried] = b;
            rep->seconds[tried] = s == TF_OK ? t : -1.0;
        }
        ++tried;
        release(p);
        if (s != TF_OK) continue;
        if (t < best_t) {
            best_t = t;
            best = b;
        }
    }
    cudaFree(dphi);
    release(qs);
    if (rep) {
        rep->n_candidates = std::min(tried, 8);
        rep->chosen = best;
        rep->cached = 0;
        rep->sample_directions = Ds;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = best;
    }
    *out = best;
    return TF_OK;
}

}  // namespace tf
