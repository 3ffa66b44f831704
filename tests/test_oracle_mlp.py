"""Pins of the learned-start oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: finite differences, invariances, saturated and
degenerate networks, the closed form of Adam under a constant gradient, exact
bfloat16 ties, a two-cell mesh worked by hand and a brute-force neighbour
search.  CPU only."""
import numpy as np
import pytest

from oracle import mlp as om
from oracle import geometry
from workloads import jittered_kuhn_mesh, random_layout


def _rand_net(I, H, O, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, om.n_params(I, H, O))


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("I,H,O,n", [(5, 8, 3, 7), (12, 16, 4, 3), (3, 8, 1, 1)])
def test_gradient_matches_central_differences(I, H, O, n):
    rng = np.random.default_rng(7 + I)
    p = _rand_net(I, H, O, 11 + H)
    X = rng.normal(0.0, 1.0, (n, I))
    T = rng.normal(0.3, 2.0, (n, O))
    mu, sd = 0.3, 1.7
    _, g = om.gradient(p, X, T, I, H, O, mu, sd)
    h = 1e-6
    fd = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (om.loss(p + e, X, T, I, H, O, mu, sd) - om.loss(p - e, X, T, I, H, O, mu, sd)) / (2 * h)
    scale = np.abs(g).max()
    assert np.abs(g - fd).max() <= 1e-7 * scale + 1e-10


def test_gradient_zero_at_exact_fit():
    """Targets equal to the network's own (de-standardised) outputs: zero loss, zero gradient."""
    I, H, O = 6, 8, 2
    p = _rand_net(I, H, O, 3)
    X = np.random.default_rng(4).normal(size=(9, I))
    y, _ = om.forward(p, X, I, H, O)
    mu, sd = -1.0, 3.0
    L, g = om.gradient(p, X, mu + sd * y, I, H, O, mu, sd)
    assert L == pytest.approx(0.0, abs=1e-28)
    assert np.abs(g).max() < 1e-14


def test_bf16_gradient_is_gradient_at_rounded_weights():
    """With bf16=True the gradient equals the plain gradient evaluated at the
    rounded weights (straight-through to the master copy)."""
    I, H, O = 4, 8, 3
    p = _rand_net(I, H, O, 5)
    W1, b1, W2, b2, W3, b3 = om.unpack(p, I, H, O)
    pr = om.pack(om.bf16_round(W1), b1, om.bf16_round(W2), b2, om.bf16_round(W3), b3)
    X = np.random.default_rng(6).normal(size=(5, I))
    T = np.random.default_rng(8).normal(size=(5, O))
    L1, g1 = om.gradient(p, X, T, I, H, O, bf16=True)
    L2, g2 = om.gradient(pr, X, T, I, H, O)
    assert L1 == L2
    assert np.array_equal(g1, g2)


# ------------------------------------------------------------------ forward
def test_forward_invariant_under_hidden_permutation():
    I, H, O = 7, 16, 5
    p = _rand_net(I, H, O, 9)
    W1, b1, W2, b2, W3, b3 = om.unpack(p, I, H, O)
    rng = np.random.default_rng(10)
    P1, P2 = rng.permutation(H), rng.permutation(H)
    q = om.pack(W1[P1], b1[P1], W2[P2][:, P1], b2[P2], W3[:, P2], b3)
    X = rng.normal(size=(11, I))
    y1, _ = om.forward(p, X, I, H, O)
    y2, _ = om.forward(q, X, I, H, O)
    np.testing.assert_allclose(y1, y2, rtol=0, atol=1e-13)
    # and a wrong permutation (columns of W2 left alone) changes the output
    q_bad = om.pack(W1[P1], b1[P1], W2[P2], b2[P2], W3[:, P2], b3)
    y3, _ = om.forward(q_bad, X, I, H, O)
    assert np.abs(y3 - y1).max() > 1e-3


def test_forward_zero_output_weights_give_bias():
    I, H, O = 5, 8, 4
    W1, b1, W2, b2, _, _ = om.unpack(_rand_net(I, H, O, 12), I, H, O)
    b3 = np.array([0.5, -2.0, 3.25, 7.0])
    p = om.pack(W1, b1, W2, b2, np.zeros((O, H)), b3)
    y, _ = om.forward(p, np.random.default_rng(1).normal(size=(6, I)), I, H, O)
    assert np.array_equal(y, np.tile(b3, (6, 1)))


def test_forward_saturated_layers():
    """Huge first-layer weights saturate tanh to the sign of W1 x; with W2 = c I the
    second layer is tanh(c) times that sign pattern, so y = tanh(c) W3 sign(W1 x) + b3."""
    I, H, O = 3, 8, 2
    rng = np.random.default_rng(13)
    W1 = rng.choice([-1.0, 1.0], size=(H, I)) * 1e3
    X = rng.choice([-1.0, 1.0], size=(4, I)) * rng.uniform(0.5, 1.0, size=(4, I))
    W1[:, 0] += 0.5e3  # keep every pre-activation away from zero
    c = 0.75
    W3 = rng.normal(size=(O, H))
    b3 = rng.normal(size=O)
    p = om.pack(W1, np.zeros(H), c * np.eye(H), np.zeros(H), W3, b3)
    y, (a1, a2) = om.forward(p, X, I, H, O)
    sgn = np.sign(X @ W1.T)
    assert np.all(np.abs(X @ W1.T) > 20)  # tanh(20) rounds to 1 in FP64
    assert np.array_equal(a1, sgn)
    np.testing.assert_allclose(y, np.tanh(c) * sgn @ W3.T + b3, rtol=0, atol=1e-14)


def test_forward_linear_regime():
    """Tiny weights: tanh(z) = z + O(z^3), so the network is the product of its
    weight matrices to third order."""
    I, H, O = 4, 8, 3
    rng = np.random.default_rng(14)
    eps = 1e-4
    W1, W2, W3 = eps * rng.normal(size=(H, I)), rng.normal(size=(H, H)) * eps, rng.normal(size=(O, H))
    p = om.pack(W1, np.zeros(H), W2, np.zeros(H), W3, np.zeros(O))
    X = rng.normal(size=(5, I))
    y, _ = om.forward(p, X, I, H, O)
    lin = X @ (W3 @ W2 @ W1).T
    assert np.abs(y - lin).max() <= 1e-6 * np.abs(lin).max()  # relative error ~ z^2 / 3


# ------------------------------------------------------------------ adam
def test_adam_constant_gradient_closed_form():
    """With a constant gradient g, m_hat = g and v_hat = g^2 at every step, so each
    step moves the parameters by exactly lr g / (|g| + eps)."""
    rng = np.random.default_rng(15)
    p0 = rng.normal(size=20)
    g = rng.normal(size=20)
    g[3] = 0.0
    m = np.zeros(20)
    v = np.zeros(20)
    p = p0.copy()
    lr = 1e-2
    for t in range(1, 6):
        p, m, v = om.adam(p, m, v, g, t, lr)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    assert p[3] == p0[3]


def test_adam_sign_flip_second_step():
    """g then -g with lr = 1, eps = 0: step 1 moves by -sign(g).  Step 2: m_2 = -0.01 g,
    v_2 = 0.001999 g^2; the bias corrections 1 - 0.9^2 = 0.19 and 1 - 0.999^2 = 0.001999
    give m_hat = -g/19, v_hat = g^2, so the move is +sign(g)/19."""
    g = np.array([2.0, -0.5])
    p, m, v = om.adam(np.zeros(2), np.zeros(2), np.zeros(2), g, 1, 1.0, eps=0.0)
    np.testing.assert_allclose(p, -np.sign(g), rtol=1e-15)
    p2, _, _ = om.adam(p, m, v, -g, 2, 1.0, eps=0.0)
    np.testing.assert_allclose(p2 - p, np.sign(g) / 19.0, rtol=1e-12)


# ------------------------------------------------------------------ bf16
def test_bf16_round_ties_and_bound():
    one = 1.0
    assert om.bf16_round(one) == 1.0
    assert om.bf16_round(1.0 + 2.0 ** -8) == 1.0                  # tie, even neighbour 1.0
    assert om.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie, even neighbour 1 + 2^-6
    assert om.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert om.bf16_round(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    assert om.bf16_round(0.0) == 0.0
    x = np.random.default_rng(16).normal(size=10000) * 10.0 ** np.random.default_rng(17).uniform(-6, 6, 10000)
    r = om.bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
    # results are representable: the low 16 bits of the single are zero
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


# ------------------------------------------------------------------ features and targets
def _two_cell_mesh():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    return xyz, tets


def test_features_two_cells_by_hand():
    G = 2
    xyz, tets = _two_cell_mesh()
    geom = geometry(xyz, tets)
    sigma_t = np.array([[1.0, 2.0], [4.0, 0.5]])
    sigma_s = np.array([[[0.5, 0.25], [0.0, 1.0]], [[1.0, 2.0], [0.0, 0.25]]])
    Q = np.zeros((2, G, 4))
    Q[0, 0] = [1, 2, 3, 6]       # average 3
    Q[0, 1] = [0, 0, 0, 4]       # average 1
    Q[1, 0] = [2, 2, 2, 2]       # average 2
    X = om.features(geom["nbr"], np.array([0, 1]), sigma_t, sigma_s, Q)
    l = np.log
    e = 1e-6
    want0 = [l(1.0), l(2.0), 0.5, 0.25, 0.0, 0.5, l(3.0 + e), l(1.0 + e), l(4.0), l(0.5), l(2.0 + e), l(e)]
    want1 = [l(4.0), l(0.5), 0.25, 0.5, 0.0, 0.5, l(2.0 + e), l(e), l(1.0), l(2.0), l(3.0 + e), l(1.0 + e)]
    np.testing.assert_allclose(X[0], want0, rtol=1e-15, atol=0)
    np.testing.assert_allclose(X[1], want1, rtol=1e-15, atol=0)


def test_features_neighbour_means_brute_force():
    """Neighbour averages against a brute-force face search (cells sharing three vertices)."""
    cfg = random_layout(n=3, G=2, n_polar=2, n_az=4, layout=1)
    geom = geometry(cfg["xyz"], cfg["tets"])
    X = om.features(geom["nbr"], cfg["cell_material"], cfg["sigma_t"], cfg["sigma_s"], cfg["Q"])
    tets = cfg["tets"]
    C, G = tets.shape[0], 2
    sets = [frozenset(t) for t in tets]
    qbar = cfg["Q"].mean(axis=2)
    lst = np.log(cfg["sigma_t"])[cfg["cell_material"]]
    for c in range(C):
        nb = [d for d in range(C) if d != c and len(sets[c] & sets[d]) == 3]
        assert 1 <= len(nb) <= 4
        np.testing.assert_allclose(X[c, 2 * G + G * G:3 * G + G * G], lst[nb].mean(axis=0), rtol=1e-14)
        np.testing.assert_allclose(X[c, 3 * G + G * G:], np.log(qbar[nb].mean(axis=0) + 1e-6), rtol=1e-14)


def test_scattering_probabilities_sum_to_ratio_range():
    """Rows of sigma_s / sigma_t sum to the scattering ratio c, drawn in [0.3, 0.99]
    for the learned-start layouts (downscatter only: the upper triangle carries it)."""
    cfg = random_layout(n=3, G=4, n_polar=2, n_az=4, layout=2)
    geom = geometry(cfg["xyz"], cfg["tets"])
    X = om.features(geom["nbr"], cfg["cell_material"], cfg["sigma_t"], cfg["sigma_s"], cfg["Q"])
    G = 4
    P = X[:, G:G + G * G].reshape(-1, G, G)
    rows = P.sum(axis=2)
    assert np.all(rows >= 0.3 - 1e-12) and np.all(rows <= 0.99 + 1e-12)
    assert np.all(np.tril(P, -1) == 0.0)


def test_targets_predict_round_trip():
    rng = np.random.default_rng(18)
    phi = rng.uniform(0.0, 5.0, size=(6, 3, 4))
    phi[0, 0] = [1e-3, -1e-3, 0.0, 0.0]          # zero average
    phi[1, 2] = [-1.0, -1.0, -1.0, -1.0]         # negative average clips to 0
    T = om.targets(phi)
    assert T[0, 0] == np.log(1e-6) and T[1, 2] == np.log(1e-6)
    back = om.predict_phi(T, 0.0, 1.0)
    avg = np.maximum(phi.mean(axis=2), 0.0)
    np.testing.assert_allclose(back[:, :, 0], avg, rtol=1e-12, atol=1e-15)
    assert np.array_equal(back[..., 0], back[..., 3])
    mu, sd = om.fit_scale(T)
    np.testing.assert_allclose(om.predict_phi((T - mu) / sd, mu, sd)[:, :, 1], avg, rtol=1e-12, atol=1e-15)


def test_fit_scale_closed_form():
    mu, sd = om.fit_scale(np.array([1.0, 3.0, 5.0, 7.0]))
    assert mu == 4.0 and sd == np.sqrt(5.0)


def test_train_steps_decrease_loss_on_linear_target():
    """A network fitting a smooth target: plain Adam lowers the loss."""
    I, H, O = 3, 16, 2
    rng = np.random.default_rng(19)
    X = rng.uniform(-1, 1, (256, I))
    T = np.stack([np.sin(X[:, 0]) + X[:, 1], X[:, 2] ** 2], axis=1)
    p = _rand_net(I, H, O, 20, 0.3)
    batches = [(X[k:k + 64], T[k:k + 64]) for k in range(0, 256, 64)] * 50
    p2, losses = om.train_steps(p, batches, I, H, O, 1e-2)
    assert om.loss(p2, X, T, I, H, O) < 0.1 * om.loss(p, X, T, I, H, O)


def test_mesh_neighbours_from_jittered_mesh_are_symmetric():
    xyz, tets = jittered_kuhn_mesh(2, 99)
    nbr = geometry(xyz, tets)["nbr"]
    for c in range(tets.shape[0]):
        for n in nbr[c]:
            if n >= 0:
                assert c in nbr[n]


def test_weighted_gradient_matches_central_differences():
    I, H, O, n = 6, 8, 3, 5
    rng = np.random.default_rng(21)
    p = _rand_net(I, H, O, 22)
    X = rng.normal(size=(n, I))
    T = rng.normal(size=(n, O))
    Wt = rng.uniform(0.0, 2.0, size=(n, O))
    _, g = om.gradient(p, X, T, I, H, O, 0.5, 1.5, W=Wt)
    h = 1e-6
    fd = np.array([(om.loss(p + h * e, X, T, I, H, O, 0.5, 1.5, W=Wt) - om.loss(p - h * e, X, T, I, H, O, 0.5, 1.5,
                                                                               W=Wt)) / (2 * h)
                   for e in np.eye(p.size)])
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(g).max()


def test_weights_are_squared_fraction_of_group_max():
    phi = np.zeros((3, 2, 4))
    phi[0, 0] = 2.0       # group 0 max
    phi[1, 0] = 1.0       # half of it
    phi[2, 0] = -1.0      # clamps to 0
    phi[:, 1] = 0.0       # a group without flux
    W = om.weights(phi, 0.01)
    np.testing.assert_allclose(W[:, 0], [1.01, 0.26, 0.01], rtol=1e-15)
    np.testing.assert_allclose(W[:, 1], [0.01, 0.01, 0.01], rtol=1e-15)
    # unit weights reproduce the unweighted loss and gradient
    I, H, O = 4, 8, 2
    p = _rand_net(I, H, O, 23)
    X = np.random.default_rng(24).normal(size=(3, I))
    T = np.random.default_rng(25).normal(size=(3, O))
    L1, g1 = om.gradient(p, X, T, I, H, O)
    L2, g2 = om.gradient(p, X, T, I, H, O, W=np.ones((3, O)))
    assert L1 == L2 and np.array_equal(g1, g2)


def test_asymmetric_loss_gradient_and_limit():
    """kappa weights overshoots: central differences still pin the gradient (the
    loss is C^1 at r = 0), kappa = 1 is the symmetric loss, and a constant fitted
    to two targets by the asymmetric loss is the kappa-weighted mean (expectile)."""
    I, H, O, n = 5, 8, 2, 6
    rng = np.random.default_rng(26)
    p = _rand_net(I, H, O, 27)
    X = rng.normal(size=(n, I))
    T = rng.normal(size=(n, O))
    _, g = om.gradient(p, X, T, I, H, O, kappa=7.0)
    h = 1e-6
    fd = np.array([(om.loss(p + h * e, X, T, I, H, O, kappa=7.0) - om.loss(p - h * e, X, T, I, H, O, kappa=7.0)) / (2 * h)
                   for e in np.eye(p.size)])
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(g).max()
    L1, g1 = om.gradient(p, X, T, I, H, O)
    L2, g2 = om.gradient(p, X, T, I, H, O, kappa=1.0)
    assert L1 == L2 and np.array_equal(g1, g2)
    # a network whose output is its bias b3 (zero W3): minimise over b3 with targets {0, 1}
    W1, b1, W2, b2, _, _ = om.unpack(p, I, H, O)
    Xs = np.zeros((2, I))
    Ts = np.array([[0.0, 0.0], [1.0, 1.0]])
    kappa = 4.0
    best = None
    for c in np.linspace(0.0, 1.0, 10001):
        q = om.pack(W1, b1, W2, b2, np.zeros((O, H)), np.full(O, c))
        L = om.loss(q, Xs, Ts, I, H, O, kappa=kappa)
        if best is None or L < best[0]:
            best = (L, c)
    # stationary point: kappa c = (1 - c)  =>  c = 1 / (1 + kappa)
    assert abs(best[1] - 1.0 / (1.0 + kappa)) < 2e-4


def test_prediction_cap():
    y = np.array([[0.0, 10.0]])
    out = om.predict_phi(y, 0.0, 1.0, cap=np.log(2.0))
    np.testing.assert_allclose(out[0, :, 0], [1.0 - 1e-6, 2.0 - 1e-6], rtol=1e-15)


def test_input_scale_standardises_columns():
    rng = np.random.default_rng(28)
    X = rng.normal(3.0, 2.0, size=(500, 4))
    X[:, 2] = 7.5                     # a constant feature
    mean, inv = om.input_scale(X)
    Z = om.normalize(X, mean, inv)
    np.testing.assert_allclose(Z[:, [0, 1, 3]].mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(Z[:, [0, 1, 3]].std(axis=0), 1.0, rtol=1e-12)
    assert inv[2] == 1.0 and np.all(Z[:, 2] == 0.0)
    # closed form on two values
    m2, i2 = om.input_scale(np.array([[1.0], [5.0]]))
    assert m2[0] == 3.0 and i2[0] == 0.5


# ------------------------------------------------------------------ context inputs
def _chain_nbr(n):
    """A chain of n cells: cell c touches c - 1 and c + 1 (neighbour lists padded with -1)."""
    nbr = -np.ones((n, 4), dtype=np.int64)
    for c in range(n):
        k = 0
        for d in (c - 1, c + 1):
            if 0 <= d < n:
                nbr[c, k] = d
                k += 1
    return nbr


def test_smooth_chain_by_hand():
    nbr = _chain_nbr(3)
    v = np.array([[3.0], [0.0], [0.0]])
    np.testing.assert_allclose(om.smooth(nbr, v, 1).ravel(), [1.5, 1.0, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(om.smooth(nbr, v, 2).ravel(), [1.25, 2.5 / 3.0, 0.5], rtol=0, atol=1e-15)
    assert np.array_equal(om.smooth(nbr, v, 0), v)


def test_smooth_is_the_power_of_the_averaging_matrix():
    """t rounds of neighbour averaging = A^t v, A the row-stochastic averaging matrix of the
    cell graph, built here independently from the mesh's face neighbours."""
    xyz, tets = jittered_kuhn_mesh(2, 9)
    nbr = geometry(xyz, tets)["nbr"]
    C = len(tets)
    A = np.zeros((C, C))
    for c in range(C):
        cells = [c] + [int(n) for n in nbr[c] if n >= 0]
        A[c, cells] = 1.0 / len(cells)
    v = np.random.default_rng(2).uniform(0.0, 1.0, (C, 3))
    for t in (1, 5, 17):
        np.testing.assert_allclose(om.smooth(nbr, v, t), np.linalg.matrix_power(A, t) @ v, rtol=1e-12, atol=1e-14)


def test_smooth_constants_and_bounds():
    xyz, tets = jittered_kuhn_mesh(2, 4)
    nbr = geometry(xyz, tets)["nbr"]
    C = len(tets)
    c = np.full((C, 2), 7.25)
    np.testing.assert_allclose(om.smooth(nbr, c, 9), c, rtol=1e-15)
    v = np.random.default_rng(3).uniform(-2.0, 5.0, (C, 2))
    s = om.smooth(nbr, v, 6)
    assert np.all(s >= v.min(axis=0) - 1e-12) and np.all(s <= v.max(axis=0) + 1e-12)  # maximum principle


def test_context_features_layout_and_zero_radius():
    """Steps (0,): the context block is the cell's own log(qbar + 1e-6) and log sigma_t; later
    blocks are the smoothings of the same starting fields, in the order the steps are given."""
    cfg = random_layout(n=3, G=2, n_polar=2, n_az=4, layout=1)
    nbr = geometry(cfg["xyz"], cfg["tets"])["nbr"]
    ctx = om.context_features(nbr, cfg["cell_material"], cfg["sigma_t"], cfg["Q"], (0, 2))
    qbar = om.cell_average(cfg["Q"])
    lst = np.log(cfg["sigma_t"])[cfg["cell_material"]]
    np.testing.assert_allclose(ctx[:, 0:2], np.log(qbar + om.EPS_T), rtol=1e-15)
    np.testing.assert_allclose(ctx[:, 2:4], lst, rtol=1e-15)
    np.testing.assert_allclose(ctx[:, 4:6], np.log(om.smooth(nbr, qbar, 2) + om.EPS_T), rtol=1e-15)
    np.testing.assert_allclose(ctx[:, 6:8], om.smooth(nbr, lst, 2), rtol=1e-15)
