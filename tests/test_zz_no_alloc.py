"""The allocation-free statistics entry point (tf_integrated_flux_noalloc),
for callers that cannot allocate device memory (their device memory belongs
to another runtime's pool, or they cannot afford cudaMalloc's implicit
synchronisation).  Its output must equal what tf_source_iterate reports for
the same flux, on two calls in a row (the shared scratch array keeps the
previous call's contents).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
import paper_2510_11513_gb300 as tf  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("G", [4, 64])
def test_noalloc_flux_statistics_match_source_iteration(G):
    cfg = W.small_box(n=6, G=G, n_polar=4, n_az=8)
    prob = tf.Problem.from_config(cfg, precision=tf.TF_FP64)
    C = prob.n_cells
    phi = torch.zeros((C, G, 4), dtype=torch.float64, device="cuda")
    res = prob.source_iterate(phi, 1e-8, 200)
    assert res["converged"]
    vol = torch.from_numpy(prob.mesh.geometry()["vol"]).cuda()
    lib = tf.load()
    for call in range(2):
        out = torch.full((G, 3), -1.0, dtype=torch.float64, device="cuda")
        st = lib.tf_integrated_flux_noalloc(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(vol.data_ptr()),
                                            ctypes.c_int64(C), ctypes.c_int32(G), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == tf.TF_OK, lib.tf_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        ref = res["integrated_flux"]
        assert np.max(np.abs(o[:, 1] - ref) / np.abs(ref)) < 1e-12, call
        assert abs(o[:, 1].sum() - res["integrated_total"]) / res["integrated_total"] < 1e-12
        p = phi.cpu().numpy()
        assert np.array_equal(o[:, 0], np.abs(p).max(axis=(0, 2)))
        assert np.allclose(o[:, 2], p.sum(axis=(0, 2)), rtol=1e-12, atol=0)


def test_noalloc_rejects_too_many_groups():
    lib = tf.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = lib.tf_integrated_flux_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                        ctypes.c_int64(1), ctypes.c_int32(1025), ctypes.c_void_p(buf.data_ptr()), None)
    assert st == tf.TF_ERR_ARG
    assert b"1024" in lib.tf_last_error()
