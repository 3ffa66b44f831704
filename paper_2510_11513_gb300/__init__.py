"""tfsweep: the unstructured S_N transport sweep (upwind DG on tetrahedra,
persistent device-queue sweep) for one GB300 GPU; host geometry and sweep
graphs of trilinear hexahedra.

The compute lives in the native library built from `csrc/` (CUDA for
sm_103a plus host C++) behind the C ABI of `include/tfsweep.h`; this package
only builds, loads and calls it.  There is no CPU or Python fallback: if the
library cannot be built or loaded, `load()` raises.
"""
from .tfsweep import (TF_ERR_ARG, TF_ERR_CUDA, TF_ERR_CYCLE, TF_ERR_DEVICE, TF_ERR_MESH, TF_ERR_NOMEM,  # noqa: F401
                      TF_ERR_NOT_CONVERGED, TF_ERR_TIMEOUT, TF_FP32, TF_FP64, TF_OK, TF_PHI_DADD, TF_PHI_PAIR,
                      TF_SCHED_AMT, TF_SCHED_BSP, TF_SCHED_BSP_LAUNCH, TF_TASK_AUTO, TF_TASK_LEVELS, TF_TASK_PATCHES,
                      HexMesh, Mesh, Mlp, Problem, Quadrature, TfError, library_path, load, options, source_iterate_batch,
                      sweep_batch, tf_destroy, tf_mlp_adam_step, tf_mlp_create, tf_mlp_features, tf_mlp_features_context, tf_mlp_fit_scale,
                      tf_mlp_fit_inputs, tf_mlp_forward, tf_mlp_gradients, tf_mlp_input_scale, tf_mlp_limits, tf_mlp_params, tf_mlp_predict_phi, tf_mlp_scale, tf_mlp_shrink,
                      tf_mlp_targets, tf_mlp_train, tf_mlp_weights,
                      tf_graph_lag, tf_graph_levels, tf_graph_tasks, tf_mesh_create, tf_mesh_create_hex, tf_mesh_geometry, tf_mesh_hex_integrals, tf_problem_create, tf_problem_psi,
                      tf_problem_stats, tf_quadrature_create, tf_quadrature_get, tf_source_iterate, tf_sweep)

__all__ = [n for n in dir() if n.startswith(("tf_", "TF_")) or n in ("HexMesh", "Mesh", "Mlp", "Problem", "Quadrature", "TfError",
                                                                       "load", "library_path", "options",
                                                                       "sweep_batch", "source_iterate_batch")]
