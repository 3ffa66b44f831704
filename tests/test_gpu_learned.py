"""Learned initial flux on the GPU against the FP64 CPU oracle (oracle/mlp.py):
features, targets, forward, gradients, Adam, prediction, training, and the
learned start's effect on source iteration."""
import numpy as np
import pytest

import workloads as W
from oracle import Problem as OracleProblem
from oracle import geometry
from oracle import mlp as om

torch = pytest.importorskip("torch")
tf = pytest.importorskip("paper_2510_11513_gb300")
from paper_2510_11513_gb300 import learned as L  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _net_and_data(I, H, O, n, seed, wscale=1.0):
    rng = np.random.default_rng(seed)
    # Glorot-like scales so every layer stays in tanh's working range
    W1 = rng.uniform(-1, 1, (H, I)) * np.sqrt(6.0 / (I + H)) * wscale
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(3.0 / H) * wscale
    W3 = rng.uniform(-1, 1, (O, H)) * np.sqrt(3.0 / H)
    p = om.pack(W1, rng.normal(0, 0.1, H), W2, rng.normal(0, 0.1, H), W3, rng.normal(0, 0.1, O))
    p = p.astype(np.float32).astype(np.float64)  # the master copy is FP32
    X = rng.normal(0.0, 1.0, (n, I)).astype(np.float32)
    T = (rng.normal(0.0, 2.0, (n, O)) - 3.0).astype(np.float32)
    return p, X, T


def _gpu_net(I, H, O, p):
    net = tf.Mlp(I, H, O, seed=1)
    net.params(set=p.astype(np.float32))
    return net


SHAPES = [(320, 64, 16, 1000), (37, 16, 5, 300), (24, 8, 3, 129), (96, 32, 64, 77)]


@pytest.mark.parametrize("I,H,O,n", SHAPES)
def test_forward_matches_oracle(I, H, O, n):
    p, X, _ = _net_and_data(I, H, O, n, seed=I + H)
    net = _gpu_net(I, H, O, p)
    Xd = torch.from_numpy(X).to(DEV)
    Y = torch.empty((n, O), dtype=torch.float32, device=DEV)
    tf.tf_mlp_forward(net.h, Xd, n, Y)
    y = Y.cpu().numpy().astype(np.float64)
    ref, _ = om.forward(p, X, I, H, O, bf16=True)
    plain, _ = om.forward(p, X, I, H, O, bf16=False)
    scale = np.abs(ref).max()
    # FP32 accumulation of BF16 weights: tight against the BF16-rounded oracle
    assert np.abs(y - ref).max() <= 2e-5 * scale
    # the BF16 rounding itself: loose against the pure FP64 network
    assert np.abs(y - plain).max() <= 3e-2 * scale


@pytest.mark.parametrize("I,H,O,n", SHAPES)
def test_gradients_match_oracle(I, H, O, n):
    p, X, T = _net_and_data(I, H, O, n, seed=3 * I + H)
    net = _gpu_net(I, H, O, p)
    mu, sd = -3.0, 2.0
    net.scale(mu, sd)
    g = np.zeros(net.n_params, np.float32)
    loss = tf.tf_mlp_gradients(net.h, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), n, grad=g)
    L_ref, g_ref = om.gradient(p, X, T, I, H, O, mu, sd, bf16=True)
    assert loss == pytest.approx(L_ref, rel=2e-5)
    # per parameter block: W1 b1 W2 b2 W3 b3
    sizes = [H * I, H, H * H, H, O * H, O]
    k = 0
    for sz in sizes:
        a, b = g[k:k + sz].astype(np.float64), g_ref[k:k + sz]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, (k, sz)
        k += sz


def test_weighted_gradients_and_weights_match_oracle():
    I, H, O, n = 320, 64, 16, 513
    p, X, T = _net_and_data(I, H, O, n, seed=31)
    rng = np.random.default_rng(32)
    phi = rng.uniform(-0.05, 1.0, (n, O, 4)) ** 3
    Wd = L.flux_weights(torch.from_numpy(phi).to(DEV), O, 1e-3)
    Wref = om.weights(phi, 1e-3)
    np.testing.assert_allclose(Wd.cpu().numpy(), Wref, rtol=1e-6, atol=1e-9)
    net = _gpu_net(I, H, O, p)
    g = np.zeros(net.n_params, np.float32)
    loss = tf.tf_mlp_gradients(net.h, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), n, grad=g, W=Wd)
    W32 = Wd.cpu().numpy().astype(np.float64)
    L_ref, g_ref = om.gradient(p, X, T, I, H, O, bf16=True, W=W32)
    assert loss == pytest.approx(L_ref, rel=2e-5)
    k = 0
    for sz in [H * I, H, H * H, H, O * H, O]:
        a, b = g[k:k + sz].astype(np.float64), g_ref[k:k + sz]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, (k, sz)
        k += sz


def test_asymmetric_gradients_and_cap_match_oracle():
    I, H, O, n = 96, 32, 8, 300
    p, X, T = _net_and_data(I, H, O, n, seed=41)
    net = _gpu_net(I, H, O, p)
    mu, sd = -3.0, 2.0
    net.scale(mu, sd)
    tf.tf_mlp_limits(net.h, kappa=6.0)
    g = np.zeros(net.n_params, np.float32)
    loss = tf.tf_mlp_gradients(net.h, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), n, grad=g)
    L_ref, g_ref = om.gradient(p, X, T, I, H, O, mu, sd, bf16=True, kappa=6.0)
    assert loss == pytest.approx(L_ref, rel=2e-5)
    k = 0
    for sz in [H * I, H, H * H, H, O * H, O]:
        a, b = g[k:k + sz].astype(np.float64), g_ref[k:k + sz]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, (k, sz)
        k += sz
    # fit_scale: mean, deviation and the cap at the largest target
    Td = torch.from_numpy(T).to(DEV)
    tf.tf_mlp_fit_scale(net.h, Td, Td.numel())
    mu2, sd2 = net.scale()
    kappa, cap = tf.tf_mlp_limits(net.h)
    m_ref, s_ref = om.fit_scale(T.astype(np.float64))
    assert mu2 == pytest.approx(m_ref, rel=1e-6) and sd2 == pytest.approx(s_ref, rel=1e-6)
    assert kappa == 6.0 and cap == float(T.max())
    phi = torch.empty((n, O, 4), dtype=torch.float64, device=DEV)
    tf.tf_mlp_predict_phi(net.h, torch.from_numpy(X).to(DEV), n, phi)
    y, _ = om.forward(p, X, I, H, O, bf16=True)
    ref = om.predict_phi(y, mu2, sd2, cap=cap)
    got = phi.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(y).max() * sd2 * (ref + 1e-6) * 1.5 + 1e-300)
    assert got.max() <= np.exp(cap)
    tf.tf_mlp_shrink(net.h, 0.5)
    tf.tf_mlp_predict_phi(net.h, torch.from_numpy(X).to(DEV), n, phi)
    ref_s = om.predict_phi(y, mu2, sd2, cap=cap, shrink=0.5)
    assert np.all(np.abs(phi.cpu().numpy() - ref_s) <= 2e-5 * np.abs(y).max() * sd2 * (ref_s + 1e-6) * 1.5 + 1e-300)


def test_input_standardisation_matches_oracle():
    I, H, O, n = 320, 64, 16, 900
    p, X, T = _net_and_data(I, H, O, n, seed=51)
    rng = np.random.default_rng(52)
    X = (X * rng.uniform(0.1, 10.0, I) + rng.uniform(-20.0, 5.0, I)).astype(np.float32)
    X[:, 7] = -13.8  # a constant feature
    net = _gpu_net(I, H, O, p)
    Xd = torch.from_numpy(X).to(DEV)
    tf.tf_mlp_fit_inputs(net.h, Xd, n)
    mean, inv = tf.tf_mlp_input_scale(net.h, I)
    m_ref, i_ref = om.input_scale(X.astype(np.float64))
    np.testing.assert_allclose(mean, m_ref, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(inv, i_ref, rtol=1e-5)
    assert inv[7] == 1.0
    Xn = om.normalize(X, mean.astype(np.float64), inv.astype(np.float64))
    Y = torch.empty((n, O), dtype=torch.float32, device=DEV)
    tf.tf_mlp_forward(net.h, Xd, n, Y)
    ref, _ = om.forward(p, Xn, I, H, O, bf16=True)
    assert np.abs(Y.cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max()
    g = np.zeros(net.n_params, np.float32)
    loss = tf.tf_mlp_gradients(net.h, Xd, torch.from_numpy(T).to(DEV), n, grad=g)
    L_ref, g_ref = om.gradient(p, Xn, T, I, H, O, bf16=True)
    assert loss == pytest.approx(L_ref, rel=2e-5)
    k = 0
    for sz in [H * I, H, H * H, H, O * H, O]:
        a, b = g[k:k + sz].astype(np.float64), g_ref[k:k + sz]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, (k, sz)
        k += sz


def test_adam_step_matches_oracle():
    I, H, O, n = 64, 32, 8, 500
    p, X, T = _net_and_data(I, H, O, n, seed=5)
    net = _gpu_net(I, H, O, p)
    tf.tf_mlp_gradients(net.h, torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), n)
    lr = 1e-3
    tf.tf_mlp_adam_step(net.h, lr)
    after = net.params().astype(np.float64)
    _, g = om.gradient(p, X, T, I, H, O, bf16=True)
    ref, _, _ = om.adam(p, np.zeros_like(p), np.zeros_like(p), g, 1, lr)
    # step 1 of Adam moves by lr g / (|g| + eps): compare where |g| >> eps
    sel = np.abs(g) > 1e-5 * np.abs(g).max()
    assert sel.mean() > 0.9
    assert np.abs(after[sel] - ref[sel]).max() <= 1e-6 * lr + 2e-7 * np.abs(ref[sel]).max()
    assert np.all(np.abs(after - p) <= lr * (1 + 1e-5) + 1e-7 * np.abs(p))  # FP32 rounding of p


def test_adam_trajectory_matches_oracle():
    """Five Adam steps over fixed minibatches: the same losses as the oracle."""
    I, H, O, n = 48, 16, 4, 256
    p, X, T = _net_and_data(I, H, O, n, seed=8)
    net = _gpu_net(I, H, O, p)
    batches = [(X[k:k + 64], T[k:k + 64]) for k in range(0, n, 64)] + [(X[:100], T[:100])]
    lr = 3e-3
    losses = []
    for Xb, Tb in batches:
        losses.append(tf.tf_mlp_gradients(net.h, torch.from_numpy(Xb).to(DEV), torch.from_numpy(Tb).to(DEV),
                                          Xb.shape[0]))
        tf.tf_mlp_adam_step(net.h, lr)
    _, ref = om.train_steps(p, batches, I, H, O, lr, bf16=True)
    np.testing.assert_allclose(losses, ref, rtol=1e-4)


def test_train_reduces_loss_on_smooth_target():
    I, H, O, n = 16, 32, 4, 20000
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (n, I)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1], X[:, 2] * X[:, 3], np.cos(X[:, 4]), X[:, 5:9].sum(axis=1)],
                 axis=1).astype(np.float32)
    net = tf.Mlp(I, H, O, seed=2)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    tf.tf_mlp_fit_scale(net.h, Td, Td.numel())
    mu, sd = net.scale()
    assert mu == pytest.approx(float(T.astype(np.float64).mean()), rel=1e-5)
    assert sd == pytest.approx(float(T.astype(np.float64).std()), rel=1e-5)
    hist = tf.tf_mlp_train(net.h, Xd, Td, n, epochs=15, batch=500, lr=3e-3, seed=4)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.05 * hist[0]
    # the final loss is the oracle's loss at the trained parameters
    p = net.params().astype(np.float64)
    ref = om.loss(p, X, T, I, H, O, mu, sd, bf16=True)
    Y = torch.empty((n, O), dtype=torch.float32, device=DEV)
    tf.tf_mlp_forward(net.h, Xd, n, Y)
    r = Y.cpu().numpy() - (T - mu) / sd
    assert float(np.mean(r.astype(np.float64) ** 2)) == pytest.approx(ref, rel=1e-4)


def test_context_features_match_oracle():
    """The wider-neighbourhood inputs (tf_mlp_features_context) against the oracle's: the one-ring
    block equal to tf_mlp_features, every context block within FP32 rounding of the oracle's."""
    cfg = W.random_layout(n=4, G=3, n_polar=2, n_az=4, layout=5)
    mesh = tf.Mesh(cfg["xyz"], cfg["tets"])
    steps = (1, 3, 8)
    X = L.cell_features(mesh, cfg, context=steps).cpu().numpy()
    X1 = L.cell_features(mesh, cfg).cpu().numpy()
    G = 3
    base = G * G + 4 * G
    assert X.shape == (mesh.n_cells, base + 2 * G * len(steps))
    assert np.array_equal(X[:, :base], X1)
    geom = geometry(cfg["xyz"], cfg["tets"])
    ref = om.context_features(geom["nbr"], cfg["cell_material"], cfg["sigma_t"], cfg["Q"], steps)
    np.testing.assert_allclose(X[:, base:], ref, rtol=2e-6, atol=2e-6)


def test_features_and_targets_match_oracle():
    cfg = W.random_layout(n=5, G=4, n_polar=2, n_az=4, layout=3)
    mesh = tf.Mesh(cfg["xyz"], cfg["tets"])
    X = L.cell_features(mesh, cfg, context=()).cpu().numpy()
    geom = geometry(cfg["xyz"], cfg["tets"])
    ref = om.features(geom["nbr"], cfg["cell_material"], cfg["sigma_t"], cfg["sigma_s"], cfg["Q"])
    np.testing.assert_allclose(X, ref, rtol=1e-7, atol=1e-7)
    rng = np.random.default_rng(11)
    phi = rng.uniform(-0.1, 3.0, (mesh.n_cells, 4, 4)) ** 3
    T = L.flux_targets(torch.from_numpy(phi).to(DEV), 4).cpu().numpy()
    np.testing.assert_allclose(T, om.targets(phi), rtol=1e-7, atol=1e-7)


def test_predict_phi_matches_oracle():
    I, H, O, n = 320, 64, 16, 700
    p, X, _ = _net_and_data(I, H, O, n, seed=12, wscale=0.5)
    net = _gpu_net(I, H, O, p)
    mu, sd = -4.0, 2.5
    net.scale(mu, sd)
    phi = torch.empty((n, O, 4), dtype=torch.float64, device=DEV)
    tf.tf_mlp_predict_phi(net.h, torch.from_numpy(X).to(DEV), n, phi)
    y, _ = om.forward(p, X, I, H, O, bf16=True)
    ref = om.predict_phi(y, mu, sd)
    got = phi.cpu().numpy()
    # y within 2e-5 |y|max, amplified by sd through exp
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(y).max() * sd * (ref + 1e-6) * 1.5 + 1e-300)


def _layout(k, n=8, G=4):
    return W.random_layout(n=n, G=G, n_polar=4, n_az=8, layout=k)


def test_learned_start_gain_and_same_answer():
    """Train on converged fluxes of 48 layouts, then solve 6 held-out layouts from zero and from
    the learned start (context inputs: the network sees the sources and cross sections well beyond
    one ring of neighbours).  The learned start takes fewer iterations in total to the same 1e-6
    stopping test, and both answers agree with the tightly converged FP64 solution within the FP32
    tolerance."""
    torch.manual_seed(0)
    train = [_layout(k) for k in range(48)]
    X, T, _, infos = L.generate(train, tol=1e-6, max_iters=3000, precision=tf.TF_FP32)
    assert all(i["converged"] for i in infos)
    ls = L.LearnedStart(4, hidden=64, seed=3)
    hist = ls.fit(X, T, epochs=30, batch=1024, lr=2e-3, seed=5)
    assert hist[-1] < 0.75 * hist[0]  # training makes progress (the context inputs start it lower)
    it_zero = it_learned = 0
    for k in range(100, 106):
        cfg = _layout(k)
        p32 = tf.Problem.from_config(cfg, precision=tf.TF_FP32)
        Xh = L.cell_features(p32.mesh, cfg, context=ls.context)
        phi0 = torch.zeros((p32.n_cells, 4, 4), dtype=torch.float64, device=DEV)
        r0 = p32.source_iterate(phi0, 1e-6, 3000)
        phi1, r1 = ls.solve(p32, Xh, 1e-6, 3000)
        assert r0["converged"] and r1["converged"]
        it_zero += r0["iterations"]
        it_learned += r1["iterations"]
        p64 = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
        ref = torch.zeros_like(phi0)
        r64 = p64.source_iterate(ref, 1e-11, 6000)
        assert r64["converged"]
        scale = ref.abs().amax(dim=(0, 2), keepdim=True)
        e0 = ((phi0 - ref).abs() / scale).max().item()
        e1 = ((phi1 - ref).abs() / scale).max().item()
        assert e1 <= max(2e-5, 2.0 * e0), (k, e0, e1)
    print(f"iterations to 1e-6 over 6 held-out layouts: zero start {it_zero}, learned start {it_learned}")
    assert it_learned < it_zero, (it_learned, it_zero)


def test_learned_start_oracle_check_one_layout():
    """One held-out layout: the learned-start FP64 solve against the oracle's own
    source iteration converged tightly on the CPU."""
    train = [_layout(k, n=6) for k in range(12)]
    X, T, _, _ = L.generate(train, tol=1e-6, max_iters=3000, precision=tf.TF_FP32)
    ls = L.LearnedStart(4, hidden=32, seed=7)
    ls.fit(X, T, epochs=20, batch=512, lr=2e-3, seed=1)
    cfg = _layout(200, n=6)
    p64 = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    phi, r = ls.solve(p64, L.cell_features(p64.mesh, cfg, context=ls.context), 1e-10, 6000)
    assert r["converged"]
    ora = OracleProblem(cfg)
    phi_o, it_o, r_o = ora.source_iterate(1e-12, 8000, threads=8)
    assert r_o < 1e-12
    got = phi.cpu().numpy()
    scale = np.abs(phi_o).max(axis=(0, 2), keepdims=True)
    # a 1e-10 stopping test leaves an error of about 1e-10 rho / (1 - rho), rho < 0.99
    assert np.all(np.abs(got - phi_o) <= 1e-7 * scale)
