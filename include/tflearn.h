/*
 * tflearn — learned initial flux for source iteration (part of libtfsweep.so).
 *
 * The paper has no counterpart of this part: its source iteration (the inner
 * and outer iterations of the benchmarks, Sec. 3 and Sec. 3.6) starts from a
 * given scalar flux.  These calls train and run a small per-cell network that
 * proposes that starting flux; tf_source_iterate then runs unchanged from it,
 * with the same stopping test, so a zero start remains the plain method and
 * the converged answer does not depend on the network.
 *
 * Network: inputs (I) -> H -> H -> outputs (O), tanh on the two hidden layers,
 * identity output.  Master parameters are FP32, flat, in this order:
 *   W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O]
 * (layer l computes z = W_l a + b_l).  The forward and backward kernels read
 * the weights W1, W2, W3 rounded to BF16 (round to nearest even) and
 * accumulate in FP32; biases stay FP32.  A handle also keeps a target
 * standardisation (mu, sd): the network output y predicts (t - mu) / sd, an
 * optional input standardisation (x - mean) inv applied to the features on
 * entry (tf_mlp_fit_inputs), and
 * an upper cap on the predicted target (tf_mlp_fit_scale sets it to the
 * largest training target, so a prediction never exceeds the largest flux
 * seen in training).
 *
 * Per-cell features (tf_mlp_features), I = G^2 + 4 G for G groups, cell c of
 * material m:
 *   x[g]                  = log sigma_t[m][g]
 *   x[G + g' G + g]       = sigma_s[m][g'][g] / sigma_t[m][g']
 *   x[G + G^2 + g]        = log(qbar[c][g] + 1e-6), qbar the mean of the 4 nodal Q[c][g][i]
 *   x[2G + G^2 + g]       = mean of log sigma_t[g] over the face neighbours
 *   x[3G + G^2 + g]       = log(mean of qbar[g] over the face neighbours + 1e-6)
 * (a cell with no neighbour takes its own values in the last two blocks).
 * Targets (tf_mlp_targets): t[c][g] = log(max(mean_i phi[c][g][i], 0) + 1e-6),
 * the log of the cell-average scalar flux; tf_mlp_predict_phi inverts that map.
 *
 * Loss over n samples: L = (1 / (n O)) sum_s sum_o w_so k_so (y_so - (t_so - mu)/sd)^2,
 * with per-target weights w (all 1 when no weight array is given) and
 * k_so = kappa where the output overshoots (y_so > (t_so - mu)/sd), else 1
 * (an asymmetric least-squares loss: kappa > 1 makes the network err low).  The
 * weights of tf_mlp_weights, w = (phi / max phi)^2 + floor per group, make a
 * log-space error count as the absolute flux error it causes relative to the
 * group's largest flux, the scale of the source-iteration stopping test.
 * Optimiser: Adam with b1 = 0.9, b2 = 0.999, eps = 1e-8 and bias correction,
 * on the FP32 master parameters; the BF16 copy is refreshed after each step.
 *
 * Conventions: X, T, Y, phi and the feature inputs are device pointers
 * (cudaMalloc or torch CUDA tensors), row-major as stated; host pointers are
 * marked "host".  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Every call returns a tf_status; the handle is destroyed with tf_destroy.
 */
#ifndef TFLEARN_H
#define TFLEARN_H

#include <stdint.h>

#include "tfsweep.h"

#ifdef __cplusplus
extern "C" {
#endif

/* New network on the current CUDA device.  n_hidden in {8, 16, 32, 64},
 * 1 <= n_out <= 64, n_in >= 1.  Weights Glorot-uniform from a Mersenne twister
 * seeded with `seed`, biases zero, (mu, sd) = (0, 1).  TF_ERR_ARG on bad sizes,
 * TF_ERR_NOMEM / TF_ERR_CUDA on device failures. */
tf_status tf_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, tf_handle *out);

/* Copies the FP32 master parameters out to `get` (host, n_params floats) and/or
 * replaces them from `set` (host; also resets the Adam moments and step count).
 * Either may be NULL; *n_params (if non-NULL) receives the count. */
tf_status tf_mlp_params(tf_handle net, float *get, const float *set, int64_t *n_params);

/* Reads (mu_get, sd_get, host) and/or sets (mu_set, sd_set, host; sd > 0) the
 * target standardisation.  Any pointer may be NULL. */
tf_status tf_mlp_scale(tf_handle net, float *mu_get, float *sd_get, const float *mu_set, const float *sd_set);

/* Reads and/or sets (host pointers, any may be NULL) the overshoot weight kappa
 * (> 0, default 1: symmetric loss) and the cap on the predicted target
 * (default +infinity). */
tf_status tf_mlp_limits(tf_handle net, float *kappa_get, float *cap_get, const float *kappa_set, const float *cap_set);

/* Reads (get) and/or sets (set, in [0, 1]; default 1) the factor that multiplies
 * the predicted flux in tf_mlp_predict_phi (host pointers, either may be NULL). */
tf_status tf_mlp_shrink(tf_handle net, float *get, const float *set);

/* Sets the input standardisation from the n rows of X [n][I]: per feature the mean
 * and inv = 1 / population standard deviation (1 for a constant feature), FP64
 * sums.  Every later call that takes features (forward, gradients, training,
 * prediction) standardises them on entry.  Synchronises `stream`. */
tf_status tf_mlp_fit_inputs(tf_handle net, const float *X, int64_t n, void *stream);

/* Reads (mean_get, inv_get: host, I floats each; TF_ERR_ARG if none is set) and/or
 * sets (mean_set and inv_set together) the input standardisation. */
tf_status tf_mlp_input_scale(tf_handle net, float *mean_get, float *inv_get, const float *mean_set, const float *inv_set);

/* Sets (mu, sd) to the mean and the population standard deviation of the
 * n_values targets T (FP64 sums) and the prediction cap to their maximum.
 * Synchronises `stream`. */
tf_status tf_mlp_fit_scale(tf_handle net, const float *T, int64_t n_values, void *stream);

/* Features of every cell into X [n_cells][G^2 + 4G] (FP32).  Inputs (device):
 * cell_material [n_cells], sigma_t [M][G], sigma_s [M][G][G] (element
 * [m][g_from][g_to]), Q [n_cells][G][4], nbr [n_cells][4] (neighbour across the
 * face opposite local vertex f, -1 on the boundary; tf_mesh_geometry gives it).
 * Asynchronous on `stream`. */
tf_status tf_mlp_features(int64_t n_cells, int32_t n_groups, const int32_t *cell_material, const double *sigma_t,
                          const double *sigma_s, const double *Q, const int32_t *nbr, float *X, void *stream);

/* Features with context: the G^2 + 4G features of tf_mlp_features, then, for each of the
 * n_scales (<= 16) ascending counts t in steps (host array), the source and the total cross
 * section seen over a neighbourhood of about sqrt(t) cells: starting from qbar (the cell-average
 * source) and log sigma_t per (cell, group), t rounds of neighbour averaging (each round replaces
 * a cell's value by the mean of its own and its face neighbours' values), written as
 * log(averaged qbar + 1e-6) (G) and averaged log sigma_t (G).  X [n_cells][G^2 + 4G + 2G n_scales]
 * (FP32, device).  One ring of neighbours cannot see a source more than one cell away, and the
 * flux at a cell is set by the sources several mean free paths around it; the context widens
 * that view.  Uses stream-ordered temporary device memory (4 n_cells G doubles).  Asynchronous on
 * `stream`.  Errors: TF_ERR_ARG, TF_ERR_CUDA. */
tf_status tf_mlp_features_context(int64_t n_cells, int32_t n_groups, const int32_t *cell_material,
                                  const double *sigma_t, const double *sigma_s, const double *Q, const int32_t *nbr,
                                  int32_t n_scales, const int32_t *steps, float *X, void *stream);

/* Targets T [n_cells][G] from a scalar flux phi [n_cells][G][4] (FP64).  Asynchronous. */
tf_status tf_mlp_targets(int64_t n_cells, int32_t n_groups, const double *phi, float *T, void *stream);

/* Weights W [n_cells][G] for the loss: w[c][g] = (pbar[c][g] / max_c pbar[c][g])^2 + floor,
 * pbar = max(mean_i phi[c][g][i], 0) (floor alone where a group's maximum is 0);
 * floor >= 0.  Allocates G words of scratch; synchronises `stream`. */
tf_status tf_mlp_weights(int64_t n_cells, int32_t n_groups, const double *phi, float floor_w, float *W, void *stream);

/* Network outputs Y [n][O] for inputs X [n][I].  Asynchronous on `stream`. */
tf_status tf_mlp_forward(tf_handle net, const float *X, int64_t n, float *Y, void *stream);

/* Loss and gradient of L over the n samples (X [n][I], T [n][O], weights W [n][O]
 * or NULL) at the current parameters; the gradient (parameter order above) is kept for tf_mlp_adam_step
 * and copied to `grad` (host, n_params floats) and the loss to `loss` (host)
 * when those are non-NULL.  Synchronises `stream`. */
tf_status tf_mlp_gradients(tf_handle net, const float *X, const float *T, const float *W, int64_t n, float *grad,
                           float *loss, void *stream);

/* One Adam step with learning rate lr > 0 from the last computed gradient.
 * Synchronises `stream`. */
tf_status tf_mlp_adam_step(tf_handle net, float lr, void *stream);

/* Minibatch training: `epochs` passes over the n samples (X, T and the optional
 * weights W as for tf_mlp_gradients), each pass over a
 * fresh shuffle (Mersenne twister seeded with `seed`) cut into consecutive
 * minibatches of `batch` samples (the last may be shorter), one Adam step per
 * minibatch.  loss_history (host, `epochs` floats, may be NULL) receives each
 * epoch's mean loss over its minibatches' samples.  Allocates its own
 * minibatch scratch; synchronises `stream`. */
tf_status tf_mlp_train(tf_handle net, const float *X, const float *T, const float *W, int64_t n, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float *loss_history, void *stream);

/* Initial flux for source iteration: phi [n_cells][O][4] (FP64, O = groups) set
 * at every node to shrink max(exp(min(mu + sd y, cap)) - 1e-6, 0), y the network output
 * for the cell's features X [n_cells][I].  Synchronises `stream`. */
tf_status tf_mlp_predict_phi(tf_handle net, const float *X, int64_t n_cells, double *phi, void *stream);

#ifdef __cplusplus
}
#endif

#endif
