"""Learned initial flux for source iteration (include/tflearn.h).

The paper's source iteration starts from a given scalar flux; a per-cell
network trained on converged fluxes proposes that start, and the iteration
then runs unchanged with the same stopping test, so a zero start remains the
plain method and the answer does not depend on the network.

This module only moves arrays and orders calls: features, targets, training,
prediction and the solves all run in libtfsweep.so's kernels.  Device arrays
are torch CUDA tensors.
"""
from __future__ import annotations

import queue
import threading
import time

import numpy as np
import torch

from . import tfsweep as tf


# Context radii of the default features: rounds of neighbour averaging (a value spreads over
# about sqrt(t) cells), so the network sees the sources and cross sections up to about 32 cells away.
CONTEXT_STEPS = (4, 16, 64, 256, 1024)


def n_features(n_groups: int, context=()) -> int:
    """Inputs per cell: log sigma_t (G), scattering probabilities (G^2), log of the
    cell-average source (G) and the face-neighbour means of log sigma_t and (log of
    the mean) of the source (2G); then 2G context inputs per entry of `context`."""
    return n_groups * n_groups + 4 * n_groups + 2 * n_groups * len(context)


def cell_features(mesh: tf.Mesh, cfg: dict, device="cuda", stream=None, context=()) -> torch.Tensor:
    """Features [n_cells][n_features(G, context)] (FP32, device) of a problem given by its mesh
    and its material / source arrays (cfg keys cell_material, sigma_t, sigma_s, Q); `context`:
    ascending rounds of neighbour averaging of the wider-neighbourhood inputs (none: one ring)."""
    G = int(cfg["n_groups"])
    C = mesh.n_cells
    nbr = torch.from_numpy(np.ascontiguousarray(mesh.geometry()["nbr"], dtype=np.int32)).to(device)
    mat = torch.from_numpy(np.ascontiguousarray(cfg["cell_material"], dtype=np.int32)).to(device)
    st = torch.from_numpy(np.ascontiguousarray(cfg["sigma_t"], dtype=np.float64)).to(device)
    ss = torch.from_numpy(np.ascontiguousarray(cfg["sigma_s"], dtype=np.float64)).to(device)
    Q = torch.from_numpy(np.ascontiguousarray(cfg["Q"], dtype=np.float64)).to(device)
    X = torch.empty((C, n_features(G, context)), dtype=torch.float32, device=device)
    if context:
        tf.tf_mlp_features_context(C, G, mat, st, ss, Q, nbr, list(context), X, stream)
    else:
        tf.tf_mlp_features(C, G, mat, st, ss, Q, nbr, X, stream)
    return X


def flux_targets(phi: torch.Tensor, n_groups: int, stream=None) -> torch.Tensor:
    """Targets [n_cells][G] (FP32): log(max(cell-average phi, 0) + 1e-6)."""
    C = phi.shape[0]
    T = torch.empty((C, n_groups), dtype=torch.float32, device=phi.device)
    tf.tf_mlp_targets(C, n_groups, phi, T, stream)
    return T


def flux_weights(phi: torch.Tensor, n_groups: int, floor: float, stream=None) -> torch.Tensor:
    """Loss weights [n_cells][G] (FP32): (cell-average phi / group maximum)^2 + floor."""
    C = phi.shape[0]
    W = torch.empty((C, n_groups), dtype=torch.float32, device=phi.device)
    tf.tf_mlp_weights(C, n_groups, phi, floor, W, stream)
    return W


def _prefetched(items, depth):
    """The items of an iterable, produced `depth` ahead by a background thread (configurations
    are built with numpy while the GPU solves the previous ones)."""
    q = queue.Queue(maxsize=max(1, depth))
    end = object()

    def produce():
        try:
            for it in items:
                q.put(it)
        except BaseException as e:  # noqa: BLE001  re-raised in the consumer
            q.put(e)
        q.put(end)

    t = threading.Thread(target=produce, daemon=True)
    t.start()
    while True:
        it = q.get()
        if it is end:
            break
        if isinstance(it, BaseException):
            raise it
        yield it
    t.join()


def generate(cfgs, tol=1e-6, max_iters=5000, device="cuda", weight_floor=None, context=CONTEXT_STEPS,
             sample_cells=0, seed=0, batch=1, **solver_opts):
    """Training data from the plain solver: for each problem configuration (any iterable; it is
    read by a background thread, `batch` ahead), its features and the targets of its converged
    zero-start solution, and with `weight_floor` the loss weights of each problem's flux.
    sample_cells > 0 keeps a seeded random subset of that many cells per problem (many layouts in
    bounded memory); batch > 1 solves that many problems together in shared launches.
    Returns (X [samples][I], T [samples][G], W [samples][G] or None, per-problem info dicts)."""
    Xs, Ts, Ws, infos = [], [], [], []
    gen = torch.Generator(device="cpu")
    gen.manual_seed(int(seed))
    pending = []

    def solve(chunk):
        t0 = time.perf_counter()
        probs = [tf.Problem.from_config(c, **solver_opts) for c in chunk]
        t_setup = (time.perf_counter() - t0) / len(chunk)
        feats = [cell_features(p.mesh, c, device, context=context) for p, c in zip(probs, chunk)]
        phis = [torch.zeros((p.n_cells, p.n_groups, 4), dtype=torch.float64, device=device) for p in probs]
        t0 = time.perf_counter()
        if len(probs) == 1:
            rs = [probs[0].source_iterate(phis[0], tol, max_iters)]
        else:
            _, rs = tf.source_iterate_batch(probs, phis, tol, max_iters)
        torch.cuda.synchronize()
        t_solve = (time.perf_counter() - t0) / len(probs)
        for prob, c, X, phi, r in zip(probs, chunk, feats, phis, rs):
            r["solve_seconds"] = t_solve
            r["setup_seconds"] = t_setup
            r["name"] = c.get("name", "")
            T = flux_targets(phi, prob.n_groups)
            Wt = flux_weights(phi, prob.n_groups, weight_floor) if weight_floor is not None else None
            if 0 < sample_cells < prob.n_cells:
                keep = torch.randperm(prob.n_cells, generator=gen)[:sample_cells].to(device)
                X, T = X[keep], T[keep]
                Wt = Wt[keep] if Wt is not None else None
            Xs.append(X)
            Ts.append(T)
            if Wt is not None:
                Ws.append(Wt)
            infos.append(r)
            prob.close()

    for cfg in _prefetched(cfgs, 2 * max(1, int(batch))):
        pending.append(cfg)
        if len(pending) == max(1, int(batch)):
            solve(pending)
            pending = []
    if pending:
        solve(pending)
    return torch.cat(Xs), torch.cat(Ts), (torch.cat(Ws) if Ws else None), infos


class LearnedStart:
    """A network mapping cell features to the initial scalar flux."""

    def __init__(self, n_groups: int, hidden: int = 64, seed: int = 0, overshoot_weight: float = 1.0,
                 shrink: float = 1.0, context=CONTEXT_STEPS):
        """overshoot_weight > 1 weights overshooting outputs more in the loss, so the
        network errs low; `shrink` scales the predicted flux (a start uniformly too low by a
        factor keeps that error in the slowest-decaying mode of source iteration, so the
        default leaves the prediction as it is); `context`: the wider-neighbourhood inputs
        (cell_features), () for one ring of neighbours only."""
        self.n_groups = int(n_groups)
        self.context = tuple(context)
        self.net = tf.Mlp(n_features(self.n_groups, self.context), hidden, self.n_groups, seed)
        tf.tf_mlp_limits(self.net.h, kappa=overshoot_weight)
        tf.tf_mlp_shrink(self.net.h, shrink)

    def fit(self, X: torch.Tensor, T: torch.Tensor, W: torch.Tensor | None = None, epochs: int = 20,
            batch: int = 1024, lr: float = 1e-3, seed: int = 0, decay: int = 3, stream=None) -> np.ndarray:
        """Standardises the inputs (per feature over X) and the targets (mean /
        standard deviation over T; predictions are capped at the largest target)
        and trains with Adam, optionally weighted by W; the epochs are split into `decay`
        phases whose learning rate drops by 3x each.  Returns the per-epoch mean loss."""
        if X.shape[0] != T.shape[0] or T.shape[1] != self.n_groups:
            raise ValueError("X and T disagree in samples or groups")
        if X.shape[1] != n_features(self.n_groups, self.context):
            raise ValueError("X does not have this network's inputs (one ring or context)")
        if W is not None and W.shape != T.shape:
            raise ValueError("W and T disagree in shape")
        tf.tf_mlp_fit_inputs(self.net.h, X, X.shape[0], stream)
        tf.tf_mlp_fit_scale(self.net.h, T, T.numel(), stream)
        phases = max(1, min(int(decay), int(epochs)))
        hist = []
        for k in range(phases):
            ep = epochs // phases + (1 if k < epochs % phases else 0)
            hist.append(tf.tf_mlp_train(self.net.h, X, T, X.shape[0], ep, batch, lr / 3.0 ** k, seed + k, W=W,
                                        stream=stream))
        return np.concatenate(hist)

    def initial_flux(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        """phi0 [n_cells][G][4] (FP64, device) for the cells whose features are X
        (cell_features with this network's context)."""
        phi = torch.empty((X.shape[0], self.n_groups, 4), dtype=torch.float64, device=X.device)
        tf.tf_mlp_predict_phi(self.net.h, X, X.shape[0], phi, stream)
        return phi

    def solve(self, problem: tf.Problem, X: torch.Tensor, tol: float, max_iters: int, stream=None):
        """Source iteration of `problem` from the learned start; returns (phi, info),
        info with the network's time as predict_seconds."""
        t0 = time.perf_counter()
        phi = self.initial_flux(X, stream)
        t_pred = time.perf_counter() - t0
        r = problem.source_iterate(phi, tol, max_iters, stream)
        r["predict_seconds"] = t_pred
        return phi, r
