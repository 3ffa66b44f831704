"""Plain FP64 CPU oracle for the learned initial flux.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
bench's CPU-baseline / reference leg may import this module.  It shares no code
with the CUDA library and never imports it.

The paper has no learned start: its source iteration starts from a given flux.
This module states, in the plainest numpy, what the library's network part
computes, so that the kernels can be checked against it:

  features   per-cell inputs read from the problem (cross sections, scattering
             probabilities, cell-average source and the averages of log sigma_t
             and of the source over the face neighbours), optionally followed by
             context inputs: the source and log sigma_t averaged over wider
             neighbourhoods (repeated neighbour averaging);
  targets    log(max(cell-average phi, 0) + 1e-6), standardised by their mean
             and deviation, predictions capped at the largest target;
  weights    (cell-average phi / its group maximum)^2 + floor, per target;
  forward    tanh MLP, inputs -> H -> H -> outputs, z = W a + b per layer;
  gradient   backpropagation of the (optionally weighted, optionally
             asymmetric: kappa on overshoots) mean squared error of the
             standardised targets;
  adam       Adam with bias correction (b1 = 0.9, b2 = 0.999, eps = 1e-8);
  inputs     per-feature standardisation (x - mean) / deviation;
  predict    the inverse of the target map, copied to the 4 nodes.

`bf16=True` rounds W1, W2, W3 to bfloat16 (round to nearest even) before use,
as the kernels do; the arithmetic stays FP64.  The gradient is then taken with
respect to the rounded weights and applied to the FP32/FP64 master copy.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss pin the
gradient; permutation of the hidden units, zero output weights and saturated
tanh layers pin the forward pass; the closed form of Adam under a constant
gradient pins the optimiser; exact bfloat16 ties pin the rounding; a two-cell
mesh worked by hand and a brute-force face-neighbour search pin the features.
"""
from __future__ import annotations

import numpy as np

EPS_T = 1e-6


# ------------------------------------------------------------------ parameters
def n_params(I, H, O):
    return H * I + H + H * H + H + O * H + O


def unpack(p, I, H, O):
    """Views W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O] of the flat vector."""
    p = np.asarray(p, dtype=np.float64)
    sizes = [H * I, H, H * H, H, O * H, O]
    shapes = [(H, I), (H,), (H, H), (H,), (O, H), (O,)]
    out, k = [], 0
    for n, s in zip(sizes, shapes):
        out.append(p[k:k + n].reshape(s))
        k += n
    assert k == p.size, "parameter vector of the wrong length"
    return out


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


def bf16_round(a):
    """Rounds to the nearest bfloat16 (ties to even), returned as float64.
    bfloat16 keeps the upper 16 bits of the IEEE single; round the lower 16."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ features
def cell_average(v):
    """Mean of the 4 nodal values (the cell average of a linear function on a tet)."""
    v = np.asarray(v, dtype=np.float64)
    return 0.25 * (((v[..., 0] + v[..., 1]) + v[..., 2]) + v[..., 3])


def features(nbr, cell_material, sigma_t, sigma_s, Q):
    """Inputs [C][G^2 + 4G] of every cell, in the order
    log sigma_t (G) | sigma_s[g'][g] / sigma_t[g'] (G*G, row g') | log(qbar + 1e-6) (G) |
    neighbour mean of log sigma_t (G) | log(neighbour mean of qbar + 1e-6) (G);
    a cell without neighbours takes its own values in the last two blocks."""
    nbr = np.asarray(nbr)
    mat = np.asarray(cell_material)
    C = mat.shape[0]
    G = sigma_t.shape[1]
    log_st = np.log(sigma_t)                                    # [M][G]
    prob = sigma_s / sigma_t[:, :, None]                        # [M][g'][g]
    qbar = cell_average(Q)                                      # [C][G]
    X = np.zeros((C, G * G + 4 * G))
    for c in range(C):
        m = mat[c]
        nb = [int(n) for n in nbr[c] if n >= 0]
        X[c, :G] = log_st[m]
        X[c, G:G + G * G] = prob[m].reshape(-1)
        X[c, G + G * G:2 * G + G * G] = np.log(qbar[c] + EPS_T)
        if nb:
            X[c, 2 * G + G * G:3 * G + G * G] = np.mean([log_st[mat[n]] for n in nb], axis=0)
            X[c, 3 * G + G * G:] = np.log(np.mean([qbar[n] for n in nb], axis=0) + EPS_T)
        else:
            X[c, 2 * G + G * G:3 * G + G * G] = log_st[m]
            X[c, 3 * G + G * G:] = np.log(qbar[c] + EPS_T)
    return X


def smooth(nbr, v, steps):
    """`steps` rounds of neighbour averaging of a per-cell field v [C][G]: each round replaces a
    cell's value by the mean of its own and its face neighbours' values (a diffusion step on the
    cell graph; after t rounds a value has spread over about sqrt(t) cells)."""
    v = np.asarray(v, dtype=np.float64).copy()
    for _ in range(int(steps)):
        out = np.empty_like(v)
        for c in range(v.shape[0]):
            nb = [int(n) for n in nbr[c] if n >= 0]
            out[c] = (v[c] + sum(v[n] for n in nb)) / (1 + len(nb))
        v = out
    return v


def context_features(nbr, cell_material, sigma_t, Q, steps):
    """Context inputs [C][2 G len(steps)]: for each t in `steps` (ascending), the source and the
    total cross section seen over a neighbourhood of about sqrt(t) cells: log(smooth_t(qbar) + 1e-6)
    (G), then smooth_t(log sigma_t) (G)."""
    mat = np.asarray(cell_material)
    qbar = cell_average(Q)
    lst = np.log(sigma_t)[mat]
    blocks, done, vq, vs = [], 0, qbar.copy(), lst.copy()
    for t in steps:
        vq, vs = smooth(nbr, vq, t - done), smooth(nbr, vs, t - done)
        done = t
        blocks += [np.log(vq + EPS_T), vs]
    return np.concatenate(blocks, axis=1)


def targets(phi):
    """t[c][g] = log(max(cell-average phi, 0) + 1e-6)."""
    return np.log(np.maximum(cell_average(phi), 0.0) + EPS_T)


def weights(phi, floor):
    """w[c][g] = (pbar[c][g] / max_c pbar[c][g])^2 + floor with pbar the clamped
    cell average; floor alone in a group whose maximum is 0."""
    pbar = np.maximum(cell_average(phi), 0.0)
    m = pbar.max(axis=0)
    r = np.divide(pbar, m, out=np.zeros_like(pbar), where=m > 0)
    return r * r + floor


def predict_phi(y, mu, sd, cap=np.inf, shrink=1.0):
    """Inverse of the standardised target map at every node, the target capped
    at `cap` (the largest training target), times `shrink`: [C][G][4]."""
    v = shrink * np.maximum(np.exp(np.minimum(mu + sd * np.asarray(y, dtype=np.float64), cap)) - EPS_T, 0.0)
    return np.repeat(v[:, :, None], 4, axis=2)


def input_scale(X):
    """Per-feature mean and inv = 1 / population standard deviation (1 where the
    feature is constant: variance <= 1e-12)."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=0)
    var = np.mean((X - mean) ** 2, axis=0)
    inv = np.where(var > 1e-12, 1.0 / np.sqrt(np.maximum(var, 1e-300)), 1.0)
    return mean, inv


def normalize(X, mean, inv):
    """(x - mean) inv per feature."""
    return (np.asarray(X, dtype=np.float64) - mean) * inv


def fit_scale(T):
    """Mean and population standard deviation of the targets."""
    T = np.asarray(T, dtype=np.float64).ravel()
    mu = T.mean()
    return mu, np.sqrt(np.mean((T - mu) ** 2))


# ------------------------------------------------------------------ network
def _weights(p, I, H, O, bf16):
    W1, b1, W2, b2, W3, b3 = unpack(p, I, H, O)
    if bf16:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    return W1, b1, W2, b2, W3, b3


def forward(p, X, I, H, O, bf16=False):
    """Outputs y [n][O] and the hidden activations (a1, a2) [n][H]."""
    W1, b1, W2, b2, W3, b3 = _weights(p, I, H, O, bf16)
    X = np.asarray(X, dtype=np.float64)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    y = a2 @ W3.T + b3
    return y, (a1, a2)


def _loss_weights(r, W, kappa):
    """Per-target weight: the given one (1 without) times kappa where the output overshoots."""
    w = np.ones_like(r) if W is None else np.asarray(W, dtype=np.float64)
    return w * np.where(r > 0.0, kappa, 1.0)


def loss(p, X, T, I, H, O, mu=0.0, sd=1.0, bf16=False, W=None, kappa=1.0):
    y, _ = forward(p, X, I, H, O, bf16)
    r = y - (np.asarray(T, dtype=np.float64) - mu) / sd
    return float(np.mean(_loss_weights(r, W, kappa) * r * r))


def gradient(p, X, T, I, H, O, mu=0.0, sd=1.0, bf16=False, W=None, kappa=1.0):
    """Loss and its gradient (flat, parameter order) by backpropagation:
    dL/dy = 2 w r / (n O) (w the given weight, 1 without, times kappa where r > 0;
    the loss is continuously differentiable at r = 0); through z3 = W3 a2 + b3, a2 = tanh(z2), z2 = W2 a1 + b2,
    a1 = tanh(z1), z1 = W1 x + b1, with tanh' = 1 - tanh^2."""
    W1, b1, W2, b2, W3, b3 = _weights(p, I, H, O, bf16)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    y, (a1, a2) = forward(p, X, I, H, O, bf16)
    r = y - (np.asarray(T, dtype=np.float64) - mu) / sd
    w = _loss_weights(r, W, kappa)
    L = float(np.mean(w * r * r))
    dy = 2.0 * w * r / (n * O)             # dL/dz3   [n][O]
    gW3 = dy.T @ a2
    gb3 = dy.sum(axis=0)
    d2 = (dy @ W3) * (1.0 - a2 * a2)       # dL/dz2   [n][H]
    gW2 = d2.T @ a1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - a1 * a1)       # dL/dz1   [n][H]
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Step t (1-based) of Adam: returns the new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train_steps(p, batches, I, H, O, lr, mu=0.0, sd=1.0, bf16=False):
    """Adam over the given list of (X, T) or (X, T, W) minibatches in order;
    returns the parameters and the loss of each minibatch before its step."""
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t, b in enumerate(batches, start=1):
        X, T = b[0], b[1]
        W = b[2] if len(b) > 2 else None
        L, g = gradient(p, X, T, I, H, O, mu, sd, bf16, W)
        losses.append(L)
        p, m, v = adam(p, m, v, g, t, lr)
    return p, losses
