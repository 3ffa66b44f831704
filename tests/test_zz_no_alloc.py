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


def _call(lib, phi_ptr, vol_ptr, C, G, out_ptr):
    return lib.tf_integrated_flux_noalloc(ctypes.c_void_p(phi_ptr), ctypes.c_void_p(vol_ptr), ctypes.c_int64(C),
                                          ctypes.c_int32(G), ctypes.c_void_p(out_ptr), None)


def test_noalloc_refuses_unreachable_or_misaligned_buffers_before_launch():
    """A plain (pageable) host buffer, or a phi address that is not 16-byte aligned, is refused
    with TF_ERR_ARG on the host: nothing is launched, so no kernel can fault on it.  A
    page-locked host buffer mapped into the device is accepted and gives the device result."""
    lib = tf.load()
    C, G = 50, 3
    rng = np.random.default_rng(7)
    phi_h = rng.uniform(0.0, 1.0, (C, G, 4))
    vol_h = rng.uniform(0.5, 1.0, C)
    phi = torch.from_numpy(phi_h).cuda()
    vol = torch.from_numpy(vol_h).cuda()
    out = torch.full((G, 3), -1.0, dtype=torch.float64, device="cuda")
    # pageable host memory (numpy): refused
    assert _call(lib, phi_h.ctypes.data, vol.data_ptr(), C, G, out.data_ptr()) == tf.TF_ERR_ARG
    assert b"host" in lib.tf_last_error()
    assert _call(lib, phi.data_ptr(), vol_h.ctypes.data, C, G, out.data_ptr()) == tf.TF_ERR_ARG
    out_h = np.zeros((G, 3))
    assert _call(lib, phi.data_ptr(), vol.data_ptr(), C, G, out_h.ctypes.data) == tf.TF_ERR_ARG
    # phi one double into a device buffer: 8-byte but not 16-byte aligned: refused
    big = torch.zeros(C * G * 4 + 1, dtype=torch.float64, device="cuda")
    assert _call(lib, big.data_ptr() + 8, vol.data_ptr(), C, G, out.data_ptr()) == tf.TF_ERR_ARG
    assert b"aligned" in lib.tf_last_error()
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == -1.0)  # nothing ran
    # device buffers, then page-locked host phi: the same numbers
    assert _call(lib, phi.data_ptr(), vol.data_ptr(), C, G, out.data_ptr()) == tf.TF_OK
    torch.cuda.synchronize()
    ref = out.cpu().numpy().copy()
    phi_p = torch.from_numpy(phi_h).pin_memory()
    out2 = torch.full((G, 3), -1.0, dtype=torch.float64, device="cuda")
    assert _call(lib, phi_p.data_ptr(), vol.data_ptr(), C, G, out2.data_ptr()) == tf.TF_OK, lib.tf_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), ref)
    assert np.allclose(ref[:, 1], np.einsum("c,cgi->g", 0.25 * vol_h, phi_h), rtol=1e-13, atol=0)
