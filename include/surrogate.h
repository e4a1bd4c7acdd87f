/* surrogate.h -- C ABI of the temperature-field surrogate in libheat.so.
 *
 * The paper has no surrogate.  This is a Fourier neural operator (FNO; Li et
 * al., 2021) that maps the 7 scalars of an instance of a layered cell --
 * conductivities k[0..4] of the 5 regions, heater source q (W/m^3) and the
 * Dirichlet temperature T_D of the boundary faces marked Dirichlet -- to the
 * temperature field after `steps` ADI steps of size dt of the paper's scheme
 * (Sec. 3) from the uniform initial temperature T_init.  The method's own
 * solver (heat_batch_*) generates its training data, is its fallback and
 * judges its error.
 *
 * Network (all sizes from surr_dims; the default is 128 x 256, width 32,
 * 12 x 12 modes, 4 layers):
 *   features (16 per cell): x_m = 2 (ln k_m - ln 0.1)/(ln 400 - ln 0.1) - 1
 *     (m < 5), x_5 = 2 (q - 1e5)/(1e7 - 1e5) - 1, x_6 = (T_D - 300)/50 (these
 *     7 broadcast over the grid), 2 r_i/R - 1, 2 z_j/Z - 1, then per cell:
 *     the one-hot region of the cell (5 channels; region = the first box
 *     containing the cell centre, all 0 on void cells), x_{region} (0 on void)
 *     and x_5 on cells of heater_region (0 elsewhere)
 *   lift v_0 = P x + pb (C channels); for l < L:
 *     pre_l = K_l(v_l) + W_l v_l + wb_l, v_{l+1} = gelu(pre_l) (l < L-1) or pre_l,
 *     K_l(v) = irfft2(pad(R_l . trunc(rfft2(v)))) over (z, r), keeping
 *     kz in {0..mz-1, Nz-mz..Nz-1}, kr in {0..mr-1}, a complex C x C matrix
 *     per kept mode;
 *   h = gelu(Q1 v_L + q1b) (2C channels), u = Q2 h + q2b (2 channels),
 *   T = T_init + m (0.02 q u_0 + (T_D - T_init) u_1)   (the scheme is linear
 *     in its source and its Dirichlet value; m = 1 on cells of a region box,
 *     0 on void cells, which the scheme keeps at T_init);
 *   gelu(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))).
 * Loss: mean over samples and cells of ((T - T_true)/(0.02 q))^2.
 * Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
 * cores (mma.sync m16n8k16), FP32 master weights, Adam in FP32.
 *
 * Flat parameter vector (FP32), in order: P[C][16], pb[C]; per layer l:
 * W_l[C][C], wb_l[C], Rre_l[2mz][mr][C][C], Rim_l[2mz][mr][C][C] (indexed
 * kz-index, kr, input channel, output channel); Q1[2C][C], q1b[2C],
 * Q2[2][2C], q2b[2].
 *
 * Layouts: params [B][7] doubles (k0..k4, q, T_D); fields [B][Nz][Nr]
 * floats, r fastest.  Status codes are those of heat.h. */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stddef.h>

#include "heat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct surr_ctx surr_ctx;

typedef struct {
    int Nz, Nr;  /* grid; must match the geometry's cell counts */
    int C;       /* width (channels), a multiple of 8 */
    int mz, mr;  /* kept modes: 2 mz along z, mr along r; mz <= Nz/2, mr < Nr/2 */
    int L;       /* spectral layers >= 1 */
} surr_dims;

/* geom, base: the cell (boxes, faces, boundary kinds) and its heat
 * capacities; base's k and q are replaced per instance by the parameters
 * (q goes to region heater_region only; T_D to every Dirichlet face).
 * dt, steps: the horizon the network predicts.  max_batch: largest number of
 * samples processed in one pass (sets the workspace; surr_forward splits
 * larger batches, surr_loss_grad requires B <= max_batch).  Copies everything
 * it needs.  HEAT_ERR_ARG on inconsistent sizes. */
int surr_create(const surr_dims *d, const heat_geometry *geom, const heat_materials *base,
                int heater_region, double dt, int steps, int max_batch, void *stream,
                surr_ctx **out);

/* Number of FP32 parameters. */
size_t surr_n_params(const surr_ctx *s);

/* Replace / read the FP32 master weights (n = surr_n_params); resets the
 * optimizer state on set. */
int surr_set_params(surr_ctx *s, const float *flat, size_t n, int on_device);
int surr_get_params(surr_ctx *s, float *flat, size_t n, int on_device);

/* Network forward: params [B][7] (host), T [B][Nz][Nr] floats (host or device). */
int surr_forward(surr_ctx *s, const double *params, int B, float *T, int on_device);

/* Loss and gradient for B <= max_batch samples: T_true [B][Nz][Nr] floats
 * (host or device).  loss (may be NULL) gets the mean loss; grad (may be
 * NULL) receives dL/dparams (n floats, host or device per grad_on_device).
 * The gradient stays inside for surr_adam. */
int surr_loss_grad(surr_ctx *s, const double *params, int B, const float *T_true, int true_on_device,
                   double *loss, float *grad, int grad_on_device);

/* One Adam step (bias-corrected, FP32 state) with the last surr_loss_grad
 * gradient; then the BF16 working copies are refreshed. */
int surr_adam(surr_ctx *s, double lr, double beta1, double beta2, double eps);

/* Inference checked against the solver, with fallback: run the network on B
 * samples; run the solver (FP32 batched path, the same dt and steps) on
 * n_check of them (indices (seed + i B / n_check) mod B); if any has
 * max|T_net - T_solver| > tol * max|T_solver - T_init|, run the solver on
 * all B samples and return its fields instead.  T: [B][Nz][Nr] floats (host
 * or device).  used_fallback: 1 if the solver's fields were returned;
 * max_err: the largest rise-relative error among the checked samples. */
int surr_infer_checked(surr_ctx *s, const double *params, int B, int n_check, double tol,
                       unsigned seed, float *T, int on_device, int *used_fallback, double *max_err);

/* The solver alone on B samples (FP32 batched path), for data generation and
 * as the baseline: T [B][Nz][Nr] floats (host or device). */
int surr_solve(surr_ctx *s, const double *params, int B, float *T, int on_device);

/* Train on n solver fields: params [n][7] (host), T_true [n][Nz][Nr] floats
 * on the device (e.g. from surr_solve with on_device = 1).  epochs passes
 * over the data in minibatches of batch <= max_batch samples, each pass in an
 * order drawn from a splitmix64 stream seeded by seed (Fisher-Yates); one
 * Adam step (beta1 0.9, beta2 0.999, eps 1e-8) per minibatch with learning
 * rate lr0 (lr_min_frac + (1 - lr_min_frac) (1 + cos(pi step / steps)) / 2),
 * a cosine decay from lr0 to lr_min_frac lr0 over all steps of the call.  last_epoch_loss (may be NULL): the
 * mean loss over the last pass.  Continues the optimizer state of earlier
 * calls.  HEAT_ERR_ARG on bad sizes or parameters; HEAT_ERR_NONFINITE if the
 * loss becomes NaN or Inf. */
int surr_train(surr_ctx *s, const double *params, int n, const float *T_true, int epochs, int batch,
               double lr0, double lr_min_frac, unsigned seed, double *last_epoch_loss);

/* The network's error on B samples with known fields T_true [B][Nz][Nr]
 * (host or device): errs[b] = max |T_net - T_true| / max |T_true - T_init|
 * over the cells of sample b (the rise-relative max error the fallback of
 * surr_infer_checked uses). */
int surr_errors(surr_ctx *s, const double *params, int B, const float *T_true, int true_on_device,
                double *errs);

void surr_destroy(surr_ctx *s);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_H */
