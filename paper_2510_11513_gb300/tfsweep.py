"""ctypes binding of the tfsweep C ABI (include/tfsweep.h).

Argument marshalling only: every computation happens in libtfsweep.so.  The
functions named tf_* mirror the C calls one to one; the small classes below
(Mesh, Quadrature, Problem) only own handles and convert arrays.

Arrays: host inputs are numpy arrays (converted to the C types and made
contiguous).  Scalar-flux buffers for tf_sweep / tf_source_iterate are
torch tensors (device or host, float64, shape [n_cells, n_groups, nodes], nodes = 4
for the linear element and 10 for the quadratic one) or numpy arrays (host); their
data pointers are passed through unchanged.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TF_OK, TF_ERR_ARG, TF_ERR_MESH, TF_ERR_CYCLE, TF_ERR_CUDA, TF_ERR_NOMEM, TF_ERR_TIMEOUT, \
    TF_ERR_NOT_CONVERGED, TF_ERR_DEVICE = range(9)
TF_FP32, TF_FP64 = 0, 1
TF_PHI_PAIR, TF_PHI_DADD = 0, 1
TF_SCHED_AMT, TF_SCHED_BSP, TF_SCHED_BSP_LAUNCH = 0, 1, 2
TF_TASK_AUTO, TF_TASK_LEVELS, TF_TASK_PATCHES = 0, 1, 2

SYMBOLS = (
    "tf_options_default", "tf_mesh_create", "tf_mesh_create_hex", "tf_mesh_hex_integrals", "tf_quadrature_create", "tf_problem_create", "tf_sweep",
    "tf_source_iterate", "tf_destroy", "tf_mesh_geometry", "tf_quadrature_get", "tf_graph_levels", "tf_graph_lag", "tf_graph_tasks",
    "tf_problem_psi", "tf_problem_set_reduce", "tf_problem_stats", "tf_status_string", "tf_last_error", "tf_integrated_flux_noalloc",
    # include/tflearn.h
    "tf_mlp_create", "tf_mlp_params", "tf_mlp_scale", "tf_mlp_limits", "tf_mlp_fit_inputs",
    "tf_mlp_input_scale", "tf_mlp_shrink", "tf_mlp_fit_scale", "tf_mlp_features", "tf_mlp_features_context",
    "tf_mlp_targets",
    "tf_mlp_weights", "tf_mlp_forward", "tf_mlp_gradients", "tf_mlp_adam_step", "tf_mlp_train", "tf_mlp_predict_phi",
)


class tf_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("device", C.c_int32), ("cells_per_task", C.c_int32), ("dir_chunk", C.c_int32),
        ("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32), ("wait_limit_s", C.c_double),
        ("phi_accumulate", C.c_int32), ("inject_stall", C.c_int32), ("psi_budget_gb", C.c_double),
        ("task_order", C.c_int32), ("staging", C.c_int32), ("octant_window", C.c_int32),
        ("pairing", C.c_int32), ("schedule", C.c_int32), ("order", C.c_int32),
        ("keep_ready", C.c_int32), ("task_shape", C.c_int32),
        ("residual_floor", C.c_double), ("patch_extent", C.c_double),
        ("lag_cycles", C.c_int32), ("reserved_i", C.c_int32), ("reserved_d", C.c_double * 1),
    ]


class tf_iter_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("converged", C.c_int32), ("residual", C.c_double),
        ("integrated_total", C.c_double), ("integrated_flux", C.POINTER(C.c_double)),
        ("residual_history", C.POINTER(C.c_double)), ("seconds", C.c_double), ("balance", C.c_double),
    ]


class tf_stats(C.Structure):
    _fields_ = [
        ("n_tasks", C.c_int64), ("n_units", C.c_int64), ("n_dirs", C.c_int32), ("max_level", C.c_int32),
        ("n_chunks", C.c_int32), ("grid_ctas", C.c_int32), ("warps_per_cta", C.c_int32),
        ("cells_per_task", C.c_int32), ("tasks_executed", C.c_int64), ("wait_polls", C.c_int64),
        ("wait_seconds", C.c_double), ("busy_seconds", C.c_double), ("kernel_seconds", C.c_double),
        ("mean_ready", C.c_double), ("source_event_seconds", C.c_double), ("sweep_event_seconds", C.c_double),
        ("phi_event_seconds", C.c_double), ("cum_source_event_seconds", C.c_double),
        ("cum_sweep_event_seconds", C.c_double), ("cum_phi_event_seconds", C.c_double), ("cum_steps", C.c_int64),
        ("launches_per_step", C.c_int64), ("kernel_mode", C.c_int32), ("tuned_n", C.c_int32),
        ("tuned_cached", C.c_int32), ("tuned_candidates", C.c_int32 * 8), ("tuned_seconds", C.c_double * 8),
        ("n_buckets", C.c_int32), ("tuned_pairing", C.c_int32), ("tuned_staging", C.c_int32),
        ("tuned_window", C.c_int32), ("task_shape", C.c_int32), ("data_wait_seconds", C.c_double),
        ("lagged_faces", C.c_int64), ("reserved_d", C.c_double * 4),
    ]


# tf_reduce_fn: int32_t (*)(void *user, double *buf, int64_t count, void *stream)
REDUCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p)


class TfError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_name(status)}) {detail}".strip())


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libtfsweep.so; builds it first if it is missing (needs nvcc).
    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"tfsweep: native library missing at {path}")
    lib = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    H = C.c_void_p
    lib.tf_options_default.argtypes = [C.POINTER(tf_options)]
    lib.tf_options_default.restype = None
    lib.tf_mesh_create.argtypes = [i64, vp, i64, vp, C.POINTER(H)]
    lib.tf_mesh_create_hex.argtypes = [i64, vp, i64, vp, C.POINTER(H)]
    lib.tf_mesh_hex_integrals.argtypes = [H, vp, vp, vp]
    lib.tf_quadrature_create.argtypes = [i32, i32, i32, vp, vp, C.POINTER(H)]
    lib.tf_problem_create.argtypes = [H, H, i32, i32, vp, vp, vp, vp, vp, vp, C.POINTER(tf_options), C.POINTER(H)]
    lib.tf_sweep.argtypes = [C.POINTER(H), i32, C.POINTER(vp), C.POINTER(vp), vp]
    lib.tf_source_iterate.argtypes = [C.POINTER(H), i32, dp, i32, C.POINTER(vp), C.POINTER(tf_iter_info), vp]
    lib.tf_destroy.argtypes = [H]
    lib.tf_mesh_geometry.argtypes = [H, C.POINTER(i64), C.POINTER(i64), vp, vp, vp, vp]
    lib.tf_quadrature_get.argtypes = [H, C.POINTER(i32), vp, vp]
    lib.tf_graph_levels.argtypes = [H, H, vp, vp]
    lib.tf_graph_lag.argtypes = [H, H, vp, vp, vp]
    lib.tf_graph_tasks.argtypes = [H, H, C.POINTER(tf_options), i32, C.POINTER(i64), vp, vp, vp]
    lib.tf_problem_psi.argtypes = [H, i32, vp, vp]
    lib.tf_problem_stats.argtypes = [H, C.POINTER(tf_stats)]
    lib.tf_problem_set_reduce.argtypes = [H, REDUCE_FN, vp]
    lib.tf_integrated_flux_noalloc.argtypes = [vp, vp, i64, i32, vp, vp]
    f32, u64, fp = C.c_float, C.c_uint64, C.POINTER(C.c_float)
    lib.tf_mlp_create.argtypes = [i32, i32, i32, u64, C.POINTER(H)]
    lib.tf_mlp_params.argtypes = [H, vp, vp, C.POINTER(i64)]
    lib.tf_mlp_scale.argtypes = [H, fp, fp, fp, fp]
    lib.tf_mlp_limits.argtypes = [H, fp, fp, fp, fp]
    lib.tf_mlp_fit_inputs.argtypes = [H, vp, i64, vp]
    lib.tf_mlp_shrink.argtypes = [H, fp, fp]
    lib.tf_mlp_input_scale.argtypes = [H, vp, vp, vp, vp]
    lib.tf_mlp_fit_scale.argtypes = [H, vp, i64, vp]
    lib.tf_mlp_features.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.tf_mlp_features_context.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp]
    lib.tf_mlp_targets.argtypes = [i64, i32, vp, vp, vp]
    lib.tf_mlp_forward.argtypes = [H, vp, i64, vp, vp]
    lib.tf_mlp_weights.argtypes = [i64, i32, vp, f32, vp, vp]
    lib.tf_mlp_gradients.argtypes = [H, vp, vp, vp, i64, vp, fp, vp]
    lib.tf_mlp_adam_step.argtypes = [H, f32, vp]
    lib.tf_mlp_train.argtypes = [H, vp, vp, vp, i64, i32, i32, f32, u64, vp, vp]
    lib.tf_mlp_predict_phi.argtypes = [H, vp, i64, vp, vp]
    lib.tf_status_string.argtypes = [i32]
    lib.tf_status_string.restype = C.c_char_p
    lib.tf_last_error.argtypes = []
    lib.tf_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        f = getattr(lib, name)
        if f.restype is C.c_int:  # default restype: the status enum
            f.restype = C.c_int
    _lib = lib
    return lib


def _status_name(s):
    try:
        return load(False).tf_status_string(s).decode()
    except Exception:  # pragma: no cover
        return str(s)


def _check(status, where):
    if status != TF_OK:
        detail = load().tf_last_error().decode()
        raise TfError(status, where, detail)
    return status


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def options(**kw) -> tf_options:
    o = tf_options()
    load().tf_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------- raw calls
def tf_mesh_create(xyz, tets):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    h = C.c_void_p()
    _check(load().tf_mesh_create(xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets), C.byref(h)), "tf_mesh_create")
    return h


def tf_mesh_create_hex(xyz, hexes):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    hexes = np.ascontiguousarray(hexes, dtype=np.int32)
    h = C.c_void_p()
    _check(load().tf_mesh_create_hex(xyz.shape[0], _ptr(xyz), hexes.shape[0], _ptr(hexes), C.byref(h)),
           "tf_mesh_create_hex")
    return h


def tf_mesh_hex_integrals(mesh, n_cells):
    out = dict(mass=np.zeros((n_cells, 8, 8)), grad=np.zeros((n_cells, 3, 8, 8)),
               face=np.zeros((n_cells, 6, 3, 4, 4)))
    _check(load().tf_mesh_hex_integrals(mesh, _ptr(out["mass"]), _ptr(out["grad"]), _ptr(out["face"])),
           "tf_mesh_hex_integrals")
    return out


def tf_quadrature_create(n_polar=0, n_azimuthal=0, omega=None, w=None):
    h = C.c_void_p()
    if omega is not None:
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        _check(load().tf_quadrature_create(0, 0, omega.shape[0], _ptr(omega), _ptr(w), C.byref(h)),
               "tf_quadrature_create")
    else:
        _check(load().tf_quadrature_create(n_polar, n_azimuthal, 0, None, None, C.byref(h)), "tf_quadrature_create")
    return h


def tf_problem_create(mesh, quad, n_groups, n_materials, cell_material, sigma_t, sigma_s, Q, S1=None,
                      psi_inflow=None, opt=None):
    cm = np.ascontiguousarray(cell_material, dtype=np.int32)
    st = np.ascontiguousarray(sigma_t, dtype=np.float64)
    ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
    Qa = np.ascontiguousarray(Q, dtype=np.float64)
    S1a = None if S1 is None else np.ascontiguousarray(S1, dtype=np.float64)
    pia = None if psi_inflow is None else np.ascontiguousarray(psi_inflow, dtype=np.float64)
    h = C.c_void_p()
    o = opt if opt is not None else options()
    _check(load().tf_problem_create(mesh, quad, int(n_groups), int(n_materials), _ptr(cm), _ptr(st), _ptr(ss),
                                    _ptr(Qa), _ptr(S1a), _ptr(pia), C.byref(o), C.byref(h)), "tf_problem_create")
    return h


def tf_sweep(problems, phi_in, phi_out, stream=None):
    n = len(problems)
    hs = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in problems])
    pin = (C.c_void_p * n)(*[_ptr(x) for x in phi_in])
    pout = (C.c_void_p * n)(*[_ptr(x) for x in phi_out])
    return _check(load().tf_sweep(hs, n, pin, pout, _stream_handle(stream)), "tf_sweep")


def tf_source_iterate(problems, tol, max_iters, phi, infos=None, stream=None):
    n = len(problems)
    hs = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in problems])
    ph = (C.c_void_p * n)(*[_ptr(x) for x in phi])
    arr = (tf_iter_info * n)(*(infos or [tf_iter_info() for _ in range(n)]))
    st = load().tf_source_iterate(hs, n, float(tol), int(max_iters), ph, arr, _stream_handle(stream))
    if st not in (TF_OK, TF_ERR_NOT_CONVERGED):
        _check(st, "tf_source_iterate")
    return st, list(arr)


def tf_destroy(h):
    return _check(load().tf_destroy(h), "tf_destroy")


def tf_mesh_geometry(mesh, n_faces=4):
    """n_faces: 4 for a tetrahedral mesh, 6 for a hexahedral one."""
    nc, nv = C.c_int64(), C.c_int64()
    _check(load().tf_mesh_geometry(mesh, C.byref(nc), C.byref(nv), None, None, None, None), "tf_mesh_geometry")
    C_, nf = nc.value, int(n_faces)
    out = dict(vol=np.zeros(C_), normal=np.zeros((C_, nf, 3)), nbr=np.zeros((C_, nf), np.int32),
               nbr_node=np.zeros((C_, nf, 4), np.int32))
    _check(load().tf_mesh_geometry(mesh, None, None, _ptr(out["vol"]), _ptr(out["normal"]), _ptr(out["nbr"]),
                                   _ptr(out["nbr_node"])), "tf_mesh_geometry")
    return out


def tf_quadrature_get(quad):
    D = C.c_int32()
    _check(load().tf_quadrature_get(quad, C.byref(D), None, None), "tf_quadrature_get")
    om = np.zeros((D.value, 3))
    w = np.zeros(D.value)
    _check(load().tf_quadrature_get(quad, None, _ptr(om), _ptr(w)), "tf_quadrature_get")
    return om, w


def tf_graph_levels(mesh, quad, n_cells, n_dirs):
    inflow = np.zeros((n_dirs, n_cells), np.uint8)
    level = np.zeros((n_dirs, n_cells), np.int32)
    _check(load().tf_graph_levels(mesh, quad, _ptr(inflow), _ptr(level)), "tf_graph_levels")
    return inflow, level


def tf_graph_lag(mesh, quad, n_cells, n_dirs):
    """(inflow, level, lag) with cycles broken by lagged back edges (tf_options.lag_cycles)."""
    inflow = np.zeros((n_dirs, n_cells), np.uint8)
    level = np.zeros((n_dirs, n_cells), np.int32)
    lag = np.zeros((n_dirs, n_cells), np.uint8)
    _check(load().tf_graph_lag(mesh, quad, _ptr(inflow), _ptr(level), _ptr(lag)), "tf_graph_lag")
    return inflow, level, lag


def tf_graph_tasks(mesh, quad, n_cells, n_dirs, n_groups, opts=None):
    """(task_of [n_dirs][n_cells], position [n_dirs][n_cells], indeg [n_tasks]) of the tasks a
    problem with these options would sweep (host only)."""
    nt = C.c_int64()
    o = opts if opts is not None else options()
    _check(load().tf_graph_tasks(mesh, quad, C.byref(o), int(n_groups), C.byref(nt), None, None, None), "tf_graph_tasks")
    task_of = np.zeros((n_dirs, n_cells), np.int32)
    position = np.zeros((n_dirs, n_cells), np.int32)
    indeg = np.zeros(nt.value, np.int32)
    _check(load().tf_graph_tasks(mesh, quad, C.byref(o), int(n_groups), C.byref(nt), _ptr(task_of), _ptr(position),
                                 _ptr(indeg)), "tf_graph_tasks")
    return task_of, position, indeg


def tf_problem_set_reduce(problem, fn):
    """fn(ptr, count, stream) -> int, or None to remove; returns the ctypes callback object, which
    the caller must keep alive while the problem may call it."""
    cb = REDUCE_FN(lambda user, buf, count, stream: int(fn(buf, count, stream))) if fn is not None else REDUCE_FN()
    _check(load().tf_problem_set_reduce(problem, cb, None), "tf_problem_set_reduce")
    return cb


def tf_problem_psi(problem, direction, out, stream=None):
    return _check(load().tf_problem_psi(problem, int(direction), _ptr(out), _stream_handle(stream)), "tf_problem_psi")


def tf_integrated_flux_noalloc(phi, volume, n_cells, n_groups, out, stream=None):
    """Per-group (max |phi|, integral, nodal sum) into `out` [n_groups, 3] (device),
    with no device allocation (see include/tfsweep.h)."""
    return _check(load().tf_integrated_flux_noalloc(_ptr(phi), _ptr(volume), int(n_cells), int(n_groups), _ptr(out),
                                                     _stream_handle(stream)), "tf_integrated_flux_noalloc")


def tf_problem_stats(problem):
    s = tf_stats()
    _check(load().tf_problem_stats(problem, C.byref(s)), "tf_problem_stats")
    out = {name: getattr(s, name) for name, _ in tf_stats._fields_ if not name.startswith("reserved")}
    out["tuned_candidates"] = list(s.tuned_candidates[: s.tuned_n])
    out["tuned_seconds"] = list(s.tuned_seconds[: s.tuned_n])
    return out


def sweep_batch(problems, phi_in, phi_out, stream=None):
    """One transport step of several problems in shared persistent launches."""
    tf_sweep([p.h for p in problems], phi_in, phi_out, stream)
    return phi_out


def source_iterate_batch(problems, phis, tol, max_iters, stream=None, history=False):
    """Source iteration of several problems in shared persistent launches; returns
    (status, [info dict per problem]) with per-problem iterations, convergence,
    residual, integrated flux and seconds to convergence."""
    infos, keep = [], []
    for p in problems:
        ig = (C.c_double * p.n_groups)()
        hist = (C.c_double * max_iters)() if history else None
        i = tf_iter_info()
        i.integrated_flux = C.cast(ig, C.POINTER(C.c_double))
        if hist is not None:
            i.residual_history = C.cast(hist, C.POINTER(C.c_double))
        infos.append(i)
        keep.append((ig, hist))
    st, out = tf_source_iterate([p.h for p in problems], tol, max_iters, phis, infos, stream)
    res = []
    for i, (ig, hist) in zip(out, keep):
        d = dict(iterations=i.iterations, converged=bool(i.converged), residual=i.residual, seconds=i.seconds,
                 integrated_total=i.integrated_total, integrated_flux=np.array(ig[:]), balance=i.balance)
        if hist is not None:
            d["residual_history"] = np.array(hist[: i.iterations])
        res.append(d)
    return st, res


# ------------------------------------------------------- learned start calls
def tf_mlp_create(n_in, n_hidden, n_out, seed=0):
    h = C.c_void_p()
    _check(load().tf_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), C.byref(h)), "tf_mlp_create")
    return h


def tf_mlp_params(net, get=None, set=None):
    n = C.c_int64()
    _check(load().tf_mlp_params(net, _ptr(get), _ptr(set), C.byref(n)), "tf_mlp_params")
    return n.value


def tf_mlp_scale(net, mu=None, sd=None):
    mu_g, sd_g = C.c_float(), C.c_float()
    mu_s = None if mu is None else C.byref(C.c_float(mu))
    sd_s = None if sd is None else C.byref(C.c_float(sd))
    _check(load().tf_mlp_scale(net, C.byref(mu_g), C.byref(sd_g), mu_s, sd_s), "tf_mlp_scale")
    return mu_g.value, sd_g.value


def tf_mlp_limits(net, kappa=None, cap=None):
    kg, cg = C.c_float(), C.c_float()
    ks = None if kappa is None else C.byref(C.c_float(kappa))
    cs = None if cap is None else C.byref(C.c_float(cap))
    _check(load().tf_mlp_limits(net, C.byref(kg), C.byref(cg), ks, cs), "tf_mlp_limits")
    return kg.value, cg.value


def tf_mlp_shrink(net, factor=None):
    g = C.c_float()
    _check(load().tf_mlp_shrink(net, C.byref(g), None if factor is None else C.byref(C.c_float(factor))),
           "tf_mlp_shrink")
    return g.value


def tf_mlp_fit_inputs(net, X, n, stream=None):
    return _check(load().tf_mlp_fit_inputs(net, _ptr(X), int(n), _stream_handle(stream)), "tf_mlp_fit_inputs")


def tf_mlp_input_scale(net, n_in, mean=None, inv=None):
    """Sets the input standardisation when mean and inv (host arrays) are given; returns (mean, inv)."""
    ms = None if mean is None else np.ascontiguousarray(mean, dtype=np.float32)
    iv = None if inv is None else np.ascontiguousarray(inv, dtype=np.float32)
    mg, ig = np.zeros(int(n_in), np.float32), np.zeros(int(n_in), np.float32)
    _check(load().tf_mlp_input_scale(net, _ptr(mg), _ptr(ig), _ptr(ms), _ptr(iv)), "tf_mlp_input_scale")
    return mg, ig


def tf_mlp_fit_scale(net, T, n_values, stream=None):
    return _check(load().tf_mlp_fit_scale(net, _ptr(T), int(n_values), _stream_handle(stream)), "tf_mlp_fit_scale")


def tf_mlp_features(n_cells, n_groups, cell_material, sigma_t, sigma_s, Q, nbr, X, stream=None):
    return _check(load().tf_mlp_features(int(n_cells), int(n_groups), _ptr(cell_material), _ptr(sigma_t),
                                         _ptr(sigma_s), _ptr(Q), _ptr(nbr), _ptr(X), _stream_handle(stream)),
                  "tf_mlp_features")


def tf_mlp_features_context(n_cells, n_groups, cell_material, sigma_t, sigma_s, Q, nbr, steps, X, stream=None):
    st = (C.c_int32 * max(1, len(steps)))(*[int(t) for t in steps])
    return _check(load().tf_mlp_features_context(int(n_cells), int(n_groups), _ptr(cell_material), _ptr(sigma_t),
                                                 _ptr(sigma_s), _ptr(Q), _ptr(nbr), len(steps), st, _ptr(X),
                                                 _stream_handle(stream)), "tf_mlp_features_context")


def tf_mlp_targets(n_cells, n_groups, phi, T, stream=None):
    return _check(load().tf_mlp_targets(int(n_cells), int(n_groups), _ptr(phi), _ptr(T), _stream_handle(stream)),
                  "tf_mlp_targets")


def tf_mlp_weights(n_cells, n_groups, phi, floor, W, stream=None):
    return _check(load().tf_mlp_weights(int(n_cells), int(n_groups), _ptr(phi), float(floor), _ptr(W),
                                        _stream_handle(stream)), "tf_mlp_weights")


def tf_mlp_forward(net, X, n, Y, stream=None):
    return _check(load().tf_mlp_forward(net, _ptr(X), int(n), _ptr(Y), _stream_handle(stream)), "tf_mlp_forward")


def tf_mlp_gradients(net, X, T, n, grad=None, W=None, stream=None):
    loss = C.c_float()
    _check(load().tf_mlp_gradients(net, _ptr(X), _ptr(T), _ptr(W), int(n), _ptr(grad), C.byref(loss),
                                   _stream_handle(stream)), "tf_mlp_gradients")
    return loss.value


def tf_mlp_adam_step(net, lr, stream=None):
    return _check(load().tf_mlp_adam_step(net, float(lr), _stream_handle(stream)), "tf_mlp_adam_step")


def tf_mlp_train(net, X, T, n, epochs, batch, lr, seed=0, W=None, stream=None):
    hist = np.zeros(int(epochs), np.float32)
    _check(load().tf_mlp_train(net, _ptr(X), _ptr(T), _ptr(W), int(n), int(epochs), int(batch), float(lr), int(seed),
                               _ptr(hist), _stream_handle(stream)), "tf_mlp_train")
    return hist


def tf_mlp_predict_phi(net, X, n_cells, phi, stream=None):
    return _check(load().tf_mlp_predict_phi(net, _ptr(X), int(n_cells), _ptr(phi), _stream_handle(stream)),
                  "tf_mlp_predict_phi")


# ------------------------------------------------------------- handle owners
class _Handle:
    h = None

    def close(self):
        if self.h is not None and _lib is not None:
            _lib.tf_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp(_Handle):
    """A per-cell network on the device (include/tflearn.h)."""

    def __init__(self, n_in, n_hidden, n_out, seed=0):
        self.h = tf_mlp_create(n_in, n_hidden, n_out, seed)
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        self.n_params = tf_mlp_params(self.h)

    def params(self, set=None):
        """The FP32 master parameters (host); replaces them first when `set` is given."""
        out = np.zeros(self.n_params, np.float32)
        tf_mlp_params(self.h, get=out, set=None if set is None else np.ascontiguousarray(set, dtype=np.float32))
        return out

    def scale(self, mu=None, sd=None):
        return tf_mlp_scale(self.h, mu, sd)


class Mesh(_Handle):
    def __init__(self, xyz, tets):
        self.h = tf_mesh_create(xyz, tets)
        self.n_cells = int(np.asarray(tets).shape[0])
        self.n_vertices = int(np.asarray(xyz).shape[0])

    def geometry(self):
        return tf_mesh_geometry(self.h)


class HexMesh(_Handle):
    """Trilinear hexahedra (tf_mesh_create_hex): host geometry, element integrals and sweep graphs."""

    def __init__(self, xyz, hexes):
        self.h = tf_mesh_create_hex(xyz, hexes)
        self.n_cells = int(np.asarray(hexes).shape[0])
        self.n_vertices = int(np.asarray(xyz).shape[0])

    def geometry(self):
        return tf_mesh_geometry(self.h, 6)

    def integrals(self):
        return tf_mesh_hex_integrals(self.h, self.n_cells)


class Quadrature(_Handle):
    def __init__(self, n_polar=0, n_azimuthal=0, omega=None, w=None):
        self.h = tf_quadrature_create(n_polar, n_azimuthal, omega, w)
        self.omega, self.w = tf_quadrature_get(self.h)
        self.n_dirs = self.omega.shape[0]


class Problem(_Handle):
    """A transport problem on the device (tf_problem_create)."""

    def __init__(self, mesh: Mesh, quad: Quadrature, n_groups, n_materials, cell_material, sigma_t, sigma_s, Q,
                 S1=None, psi_inflow=None, **opts):
        self.mesh, self.quad = mesh, quad
        self.opt = options(**opts)
        self.n_nodes = 8 if isinstance(mesh, HexMesh) else {2: 10, 3: 20}.get(int(self.opt.order), 4)
        if int(n_groups) > 0 and np.size(Q) != mesh.n_cells * int(n_groups) * self.n_nodes:
            raise ValueError(f"Q must be [n_cells][n_groups][{self.n_nodes}]")
        self.h = tf_problem_create(mesh.h, quad.h, n_groups, n_materials, cell_material, sigma_t, sigma_s, Q, S1,
                                   psi_inflow, self.opt)
        self.n_groups = int(n_groups)
        self.n_cells = mesh.n_cells
        self.n_dirs = quad.n_dirs
        self.precision = self.opt.precision

    @classmethod
    def from_config(cls, cfg, S1=None, psi_inflow=None, omega=None, w=None, **opts):
        mesh = HexMesh(cfg["xyz"], cfg["hexes"]) if "hexes" in cfg else Mesh(cfg["xyz"], cfg["tets"])
        quad = Quadrature(omega=omega, w=w) if omega is not None else Quadrature(cfg["n_polar"], cfg["n_azimuthal"])
        return cls(mesh, quad, cfg["n_groups"], cfg["n_materials"], cfg["cell_material"], cfg["sigma_t"],
                   cfg["sigma_s"], cfg["Q"], S1=S1, psi_inflow=psi_inflow, **opts)

    @property
    def n_units(self):
        return self.n_cells * self.n_dirs * self.n_groups

    def sweep(self, phi_in, phi_out, stream=None):
        tf_sweep([self.h], [phi_in], [phi_out], stream)
        return phi_out

    def source_iterate(self, phi, tol, max_iters, stream=None, history=False):
        G = self.n_groups
        ig = (C.c_double * G)()
        hist = (C.c_double * max_iters)() if history else None
        info = tf_iter_info()
        info.integrated_flux = C.cast(ig, C.POINTER(C.c_double))
        if hist is not None:
            info.residual_history = C.cast(hist, C.POINTER(C.c_double))
        st, out = tf_source_iterate([self.h], tol, max_iters, [phi], [info], stream)
        i = out[0]
        res = dict(status=st, iterations=i.iterations, converged=bool(i.converged), residual=i.residual,
                   integrated_total=i.integrated_total, integrated_flux=np.array(ig[:]), balance=i.balance)
        if hist is not None:
            res["residual_history"] = np.array(hist[: i.iterations])
        return res

    def set_reduce(self, fn):
        """Sum of the partial phi over partners (direction sharding); fn(ptr, count, stream) -> 0 on
        success.  None removes it."""
        self._reduce_cb = tf_problem_set_reduce(self.h, fn)

    def psi(self, direction, out, stream=None):
        tf_problem_psi(self.h, direction, out, stream)
        return out

    def stats(self):
        return tf_problem_stats(self.h)
