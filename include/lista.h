/* liblassogs -- learned warm start for the Lasso solver.
 *
 * The paper has no learned component.  This part only proposes the starting
 * point beta0 handed to lasso_path / lasso_batch; the solver's safety does not
 * depend on it: any beta0 yields a feasible dual point through the rescaling
 * of Eq. (8) (theta = rho / max(lambda, ||X^T rho||_inf)), and every screening
 * test (Eq. (7)) and stopping test uses the duality gap computed exactly from
 * the current iterate.  A poor beta0 costs passes, never correctness.
 *
 * Model: an unrolled ISTA network with L layers, a p x n matrix W tied over
 * the layers, per-layer elementwise steps d_l (length p) and thresholds
 * tau_l.  For a response y (length n):
 *     s = ||X^T y||_inf (lambda_max of y, Sec. 1.2),  ytil = y / s,
 *     beta^0 = 0,  for l = 0 .. L-1:
 *         u_l = ytil - X beta^l,  v_l = W u_l,  z_l = beta^l + d_l .* v_l,
 *         beta^{l+1} = ST(z_l, tau_l),  ST(z, t) = sign(z) max(|z| - t, 0),
 *     warm start beta0 = s * beta^L.
 * The Lasso solution is positively homogeneous (beta_hat(c y, c lambda) =
 * c beta_hat(y, lambda)), so one network trained on normalised responses
 * serves every y at a fixed ratio lambda / lambda_max.  With W = X^T,
 * d_l = 1/||X||_2^2 and tau_l = ratio/||X||_2^2 it is L steps of ISTA.
 *
 * Training minimises 1/(2B) sum_b ||beta^L_b - t_b||^2 over pairs
 * (ytil_b, t_b = beta_hat_b / s_b) whose beta_hat_b the solver produced.
 *
 * Precision: FP32 storage and arithmetic (products accumulated in FP32 by
 * CUDA-core GEMM kernels with fixed reduction order: results are
 * deterministic run to run); loss in FP64.
 *
 * Layouts (all device memory, caller-owned):
 *   X      FP32, column j at X + j*ldx (as for lasso_path), n x p
 *   W      p x n FP32, row j at W + j*n (the layout of X^T)
 *   D      L x p FP32, row l = d_l;   tau  L FP32
 *   per-sample vectors are rows: Ytil B x n (row b at Ytil + b*ldyt),
 *   beta, targets and gradients of beta B x p with leading dimension p.
 * Errors: LASSO_ERR_INVALID_ARG (bad sizes or NULL), LASSO_ERR_WORKSPACE
 * (workspace too small or misaligned), LASSO_ERR_CUDA (launch failure);
 * message in lasso_last_error().  Calls are asynchronous on `stream`. */
#ifndef LISTA_H
#define LISTA_H

#include <stddef.h>
#include <stdint.h>

#include "lassogs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of workspace every lista_* call below needs for these sizes (it
 * holds the per-layer cache u_l, v_l, z_l of a forward pass for the backward
 * pass, and the split-K partial sums).  0 for invalid sizes. */
size_t lista_workspace_size(int64_t n, int64_t p, int32_t L, int64_t B);

/* Where lista_forward(keep_cache = 1) leaves its per-layer cache inside the
 * workspace (for inspection): byte offsets of u_0 (B x n floats per layer,
 * layer l at off_u + 4*l*B*n), v_0 and z_0 (B x p floats per layer, layer l at
 * off + 4*l*B*p).  Rows are samples.  Returns LASSO_ERR_INVALID_ARG for bad
 * sizes or NULL outputs. */
lasso_status lista_cache_layout(int64_t n, int64_t p, int32_t L, int64_t B, int64_t* off_u, int64_t* off_v,
                                int64_t* off_z);

/* ISTA initialisation: ||X||_2^2 estimated by 60 steps of the power method
 * on X^T X (scaled up by 1 %), then W = X^T, d_l = 1/||X||_2^2,
 * tau_l = ratio/||X||_2^2.  lip_out (device, 1 float) receives the estimate,
 * may be NULL. */
lasso_status lista_init(const float* X, int64_t n, int64_t p, int64_t ldx, int32_t L, float ratio, float* W,
                        float* D, float* tau, float* lip_out, void* workspace, size_t workspace_bytes, void* stream);

/* s_b = ||X^T y_b||_inf and ytil_b = y_b / s_b (0 when s_b = 0) for the B
 * responses Y (FP64, row b at Y + b*ldy).  Outputs s (B floats) and Ytil. */
lasso_status lista_normalize(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                             int64_t B, float* Ytil, int64_t ldyt, float* s, void* workspace, size_t workspace_bytes,
                             void* stream);

/* beta^L for B normalised responses into beta_out (B x p, leading dim p).
 * keep_cache = 1 stores u_l, v_l, z_l in the workspace for lista_backward. */
lasso_status lista_forward(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                           const float* tau, int32_t L, const float* Ytil, int64_t ldyt, int64_t B, float* beta_out,
                           int32_t keep_cache, void* workspace, size_t workspace_bytes, void* stream);

/* Gradients of the loss 1/(2B) sum_b ||beta^L_b - t_b||^2 for the batch of
 * the preceding lista_forward(keep_cache = 1) on the same workspace, sizes
 * and parameters.  betaL is that call's beta_out; targets B x p.  Writes
 * gW (p x n), gD (L x p), gtau (L) and the loss (FP64, device) to loss_out.
 * The derivative of ST at |z| = tau is taken as 0. */
lasso_status lista_backward(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                            const float* tau, int32_t L, int64_t B, const float* betaL, const float* targets,
                            float* gW, float* gD, float* gtau, double* loss_out, void* workspace,
                            size_t workspace_bytes, void* stream);

/* One Adam step (Kingma & Ba, 2015, Algorithm 1) at step t >= 1 on count
 * parameters: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
lasso_status lista_adam(float* theta, const float* grad, float* m, float* v, int64_t count, int32_t t, float lr,
                        float b1, float b2, float eps, void* stream);

/* dst row r = src row idx[r] (idx device int32, B entries, each in
 * [0, rows of src)), width floats per row: assembles a minibatch. */
lasso_status lista_gather(const float* src, int64_t ld_src, const int32_t* idx, int64_t B, int64_t width,
                          float* dst, int64_t ld_dst, void* stream);

/* Training targets t_b = beta_hat_b / s_b (0 when s_b = 0) from FP64 solver
 * output (row b at beta_hat + b*ldbh) into FP32 targets (B x p, ld p). */
lasso_status lista_targets(const double* beta_hat, int64_t ldbh, const float* s, int64_t B, int64_t p,
                           float* targets, void* stream);

/* Inference: beta0_b = s_b * beta^L(ytil_b) for B responses Y (FP64, row b at
 * Y + b*ldy), written as FP64 rows of beta0 (leading dimension ldb0 >= p):
 * the layout lasso_batch takes as its starting points.
 * max_nonzeros > 0 keeps, per row, only the entries whose magnitude is among
 * the max_nonzeros largest (ties at the cut are all dropped) and sets the
 * rest to 0: a Lasso solution in general position has at most n nonzeros, and
 * coordinate descent pays per pass for every nonzero of its iterate, so a
 * dense start costs more than it saves.  max_nonzeros <= 0 keeps all. */
lasso_status lista_warm_start(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                              const float* tau, int32_t L, const double* Y, int64_t ldy, int64_t B, double* beta0,
                              int64_t ldb0, int64_t max_nonzeros, void* workspace, size_t workspace_bytes,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LISTA_H */
