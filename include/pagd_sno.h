/*
 * pagd_sno.h -- C ABI of the learned initial iterate: a small spectral neural
 * operator (FNO-style spectral layers) that proposes u^{n+1} for an implicit
 * time step, trained on trajectories the solver generates.
 *
 * The paper starts PAGD from the extrapolation x_0 = u^n + rho (u^n - u^{n-1})
 * (Sec. 3.4.2, Algorithm 2); it has no learned component.  The network here
 * predicts the correction to that extrapolation; pagd_step_with_guess (pagd.h)
 * takes the proposal and keeps it only when its first PAGD direction is
 * smaller than the extrapolation's, so the result of a step never depends on
 * the network beyond the stopping tolerance.
 *
 * Network (per sample, grid n0 x n1, np = n0 n1, C channels, L layers, kept
 * modes k0 in [-M0/2, M0/2) and k1 in [0, M1)):
 *   a = [u^n, s_in (u^n - u^{n-1})];  v_0 = P a + b_P;
 *   v_{l+1} = GELU(W_l v_l + b_l + K_l v_l);  out = Q v_L + b_Q;
 *   guess = u^n + rho (u^n - u^{n-1}) + s_out out,
 *   (K v)[o] = Re sum_m w_m (sum_c R[o][c][m] F[c][m]) e^{i k_m.x} / np,
 *   F[c][m] = sum_x v[c](x) e^{-i k_m.x},  w_m = 1 (k1 = 0) or 2.
 * Parameters: one flat FP32 device array, in order P [C][2], b_P [C]; per
 * layer W [C][C], b [C], R [C][C][M0 M1][2] (re, im); Q [C], b_Q.
 * Fields u^n, u^{n-1}, targets and guesses are FP64 device arrays of nsamples
 * x np values (sample-major).  All work runs on the stream given at creation;
 * calls that return values synchronise it.  Every call returns a pagd_status
 * (values from pagd.h) and never aborts.
 */
#ifndef PAGD_SNO_H
#define PAGD_SNO_H

#include <stddef.h>

#include "pagd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sno_net sno_net; /* opaque, library-owned host object */

/* Powers of two 8..4096 for n0, n1; channels 1..32; layers 1..16; modes0 even,
 * <= n0; modes1 <= min(32, n1/2); modes0 * modes1 <= 1024; batch >= 1 (the
 * largest nsamples of later calls). */
pagd_status sno_create(sno_net** out, int n0, int n1, int channels, int layers, int modes0, int modes1, int batch,
                       void* stream);
pagd_status sno_param_count(const sno_net* s, size_t* count);
/* Device workspace (activations kept for the backward pass): query, allocate,
 * hand in (256-byte aligned); it must stay valid while the network is used. */
pagd_status sno_workspace_size(const sno_net* s, size_t* bytes);
pagd_status sno_set_workspace(sno_net* s, void* dev_ptr, size_t bytes);

/* Inference: guess (device, nsamples x np FP64) from u^n, u^{n-1}. */
pagd_status sno_predict(sno_net* s, const float* params, const double* un, const double* unm1, double rho,
                        double s_in, double s_out, int nsamples, double* guess);

/* Training: loss = mean over samples and points of (out - t)^2 with
 * t = (target - x_0) / s_out, and its gradient with respect to every parameter
 * (grad: device FP32, param_count values, overwritten).  loss (host, nullable). */
pagd_status sno_loss_grad(sno_net* s, const float* params, const double* un, const double* unm1,
                          const double* target, double rho, double s_in, double s_out, int nsamples, float* grad,
                          double* loss);

/* One Adam update (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) of
 * params with moments m, v (device FP32, param_count each, zero at t = 1);
 * t = 1, 2, ... the update count, lr the step size. */
pagd_status sno_adam_step(sno_net* s, float* params, const float* grad, float* m, float* v, int t, double lr);

/* BF16 weights: weights[i] = master[i] rounded to the nearest BF16 value (ties
 * to even), stored as FP32 (device arrays of param_count values; may not
 * alias).  With these weights the network computes in FP32 on BF16-valued
 * parameters; training keeps the FP32 master copy for Adam and re-rounds
 * after every update. */
pagd_status sno_round_bf16(sno_net* s, const float* master, float* weights);

const char* sno_last_error(const sno_net* s);
void sno_destroy(sno_net* s);

#ifdef __cplusplus
}
#endif
#endif /* PAGD_SNO_H */
