"""Direction sharding on one GPU.  A problem on a share of the directions computes the partial
flux sum_{a in share} w_a psi_a (Eq. (2)); the shares' partial fluxes add up to the flux of the
whole set.  With a reduce function (tf_problem_set_reduce), partners iterate on the summed flux
and leakage: here two host threads stand for two processes, and their reduce function sums the
two partial device buffers between the launches (a host rendezvous, no kernel waits on another).
The sharded source iteration must reach the unsharded answer in the same number of iterations."""
import threading

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402
from paper_2510_11513_gb300 import shard  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _shard_problems(cfg, world, precision, **opts):
    om, w = oracle.product_quadrature(cfg["n_polar"], cfg["n_azimuthal"])
    out = []
    for r in range(world):
        o_r, w_r = shard.shard_quadrature(om, w, r, world)
        out.append(tf.Problem.from_config(cfg, omega=o_r, w=w_r, precision=precision, **opts))
    return out


@pytest.mark.parametrize("precision,G,tol", [(tf.TF_FP64, 32, 1e-13), (tf.TF_FP32, 64, 2e-7), (tf.TF_FP64, 5, 1e-13)])
def test_partial_fluxes_of_the_shares_add_up_to_the_whole(precision, G, tol):
    cfg = W.two_material_box(n=6, G=G, n_polar=4, n_az=8)
    full = tf.Problem.from_config(cfg, precision=precision)
    C = full.n_cells
    phi_in = torch.from_numpy(np.random.default_rng(11).uniform(0.0, 1.0, (C, G, 4))).cuda()
    ref = torch.zeros_like(phi_in)
    full.sweep(phi_in, ref)
    ref = ref.cpu().numpy()
    total = np.zeros_like(ref)
    for p in _shard_problems(cfg, 2, precision):
        out = torch.zeros_like(phi_in)
        p.sweep(phi_in, out)
        total += out.cpu().numpy()
    assert _rel(total, ref) < tol
    ora = oracle.Problem(cfg).transport_step(phi_in.cpu().numpy(), threads=8)
    assert _rel(total, ora) < (1e-11 if precision == tf.TF_FP64 else 2e-5)


class _ThreadPartners:
    """Reduce functions for `n` problems iterated by `n` host threads: each call waits for the
    other partners, sums their partial device buffers in a fixed order and writes the sum back."""

    def __init__(self, n):
        self.bar = threading.Barrier(n, timeout=120)
        self.bufs = [None] * n
        self.calls = [0] * n

    def fn(self, rank):
        def reduce(ptr, count, stream):
            torch.cuda.synchronize()
            t = torch.as_tensor(shard._DeviceBuffer(ptr, count), device="cuda")
            self.bufs[rank] = t
            self.bar.wait()
            s = self.bufs[0].clone()
            for b in self.bufs[1:]:
                s += b
            torch.cuda.synchronize()
            self.bar.wait()  # every partner has read every partial
            t.copy_(s)
            torch.cuda.synchronize()
            self.bar.wait()
            self.calls[rank] += 1
            return 0
        return reduce


@pytest.mark.parametrize("precision,G", [(tf.TF_FP64, 32), (tf.TF_FP32, 64)])
def test_sharded_source_iteration_matches_unsharded(precision, G):
    cfg = W.two_material_box(n=6, G=G, n_polar=4, n_az=8)
    tol = 1e-9 if precision == tf.TF_FP64 else 1e-6
    full = tf.Problem.from_config(cfg, precision=precision)
    C = full.n_cells
    phi_ref = torch.zeros((C, G, 4), dtype=torch.float64, device="cuda")
    r_ref = full.source_iterate(phi_ref, tol, 300)
    assert r_ref["converged"]
    world = 2
    probs = _shard_problems(cfg, world, precision)
    partners = _ThreadPartners(world)
    for r, p in enumerate(probs):
        p.set_reduce(partners.fn(r))
    phis = [torch.zeros((C, G, 4), dtype=torch.float64, device="cuda") for _ in range(world)]
    res = [None] * world
    errs = []

    def run(r):
        try:
            res[r] = probs[r].source_iterate(phis[r], tol, 300)
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)
            partners.bar.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    a = phis[0].cpu().numpy()
    assert np.array_equal(a, phis[1].cpu().numpy())  # both partners hold the same flux
    assert res[0]["iterations"] == res[1]["iterations"] == r_ref["iterations"]
    assert partners.calls[0] == 2 * res[0]["iterations"]  # the flux and the leakage, every step
    ref = phi_ref.cpu().numpy()
    assert _rel(a, ref) < (1e-12 if precision == tf.TF_FP64 else 2e-5)
    assert abs(res[0]["balance"]) < (1e-12 if precision == tf.TF_FP64 else 1e-5)
    assert np.allclose(res[0]["integrated_flux"], r_ref["integrated_flux"], rtol=1e-10 if precision == tf.TF_FP64 else 2e-5)


def test_reduce_function_errors():
    cfg = W.two_material_box(n=3, G=32, n_polar=2, n_az=4)
    p = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    q = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    phi = torch.zeros((p.n_cells, 32, 4), dtype=torch.float64, device="cuda")
    p.set_reduce(lambda ptr, count, stream: 3)
    with pytest.raises(tf.TfError) as e:
        p.source_iterate(phi, 1e-6, 5)
    assert e.value.status == tf.TF_ERR_CUDA
    with pytest.raises(tf.TfError) as e:
        tf.source_iterate_batch([p, q], [phi, torch.zeros_like(phi)], 1e-6, 5)
    assert e.value.status == tf.TF_ERR_ARG
    p.set_reduce(None)  # removed: the problem iterates on its own again
    assert p.source_iterate(phi, 1e-6, 100)["converged"]
