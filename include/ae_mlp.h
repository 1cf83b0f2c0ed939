/*
 * ae_mlp.h — C ABI of the search-work predictor in libae.so.
 *
 * The predictor is not part of the paper's method and never changes a search
 * result.  For a DNA query it estimates two numbers of the query's search:
 * y0 = log1p(DP entries computed) and y1 = log1p(raw hits written by the
 * text-position sweep), from 66 features of the query.  Callers use the
 * estimates to size buffers (ae_options.hint_hits), to pack queries into
 * batches and to admit requests by device memory.
 *
 * Features (ae_mlp_features), per query of m letters:
 *   f[0..63]  3-mer spectrum: occurrences of 3-mer (a,b,c) -- index 16a+4b+c,
 *             letters in ACGT order -- divided by the m-2 windows (0 if m<3);
 *   f[64]     log1p(m);
 *   f[65]     the mean, over the query's m-K+1 windows of K letters, of
 *             log1p(|SA interval of the window|), K = ceil(log4(n+1)) + 4 for
 *             a text of n letters (0 if m < K); the interval size is the
 *             number of occurrences of the window in the text (Section 2.3:
 *             one suffix-array row per occurrence), taken from the FM index
 *             by K backward steps (Section 5 (3)).  Windows of an unrelated
 *             query are rarely found at this length, those of a query with
 *             homologs in the text often are.
 *
 * Network: y = W3 relu(W2 relu(W1 x' + b1) + b2) + b3 with sizes
 * 66-128-128-2, x' = (f - x_mu) / x_sd, and the output mapped back as
 * y * y_sd + y_mu.  Parameters are kept in fp32 (packed in the order W1
 * [128x66 row-major], b1[128], W2[128x128], b2[128], W3[2x128], b3[2]; 25,346
 * floats); every matrix product rounds its operands to bfloat16 and
 * accumulates in fp32 on the tensor cores (mma.sync m16n8k16 bf16).
 * Training minimises L = sum((y' - t')^2) / (2B) over a batch, t' = (t - y_mu)
 * / y_sd, with Adam (beta1 0.9, beta2 0.999, eps 1e-8) and decoupled weight
 * decay: p -= lr * (m_hat / (sqrt(v_hat) + eps) + weight_decay * p).
 *
 * All device arrays are fp32 row-major on the current device; a model is used
 * by one thread at a time.  Errors: AE_EINVAL (bad sizes or NULL), AE_ENOMEM,
 * AE_ECUDA, AE_EUNSUPPORTED (features of a non-DNA index).
 */
#ifndef AE_MLP_H
#define AE_MLP_H

#include <stdint.h>

#include "ae.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ae_mlp ae_mlp;

enum { AE_MLP_IN = 66, AE_MLP_HIDDEN = 128, AE_MLP_OUT = 2, AE_MLP_PARAMS = 25346 };

/* New model with He-uniform weights drawn from `seed`, zero biases and
 * identity normalisation, on the current device. */
ae_status ae_mlp_create(uint64_t seed, ae_mlp **out);
void ae_mlp_free(ae_mlp *mlp);

/* Copy the packed parameters (host, AE_MLP_PARAMS floats) in or out.  Setting
 * parameters also resets Adam's moments and step count. */
ae_status ae_mlp_set_params(ae_mlp *mlp, const float *params);
ae_status ae_mlp_get_params(const ae_mlp *mlp, float *params);

/* Input and output normalisation (host arrays of 66, 66, 2, 2 floats; every
 * sd must be > 0). */
ae_status ae_mlp_set_norm(ae_mlp *mlp, const float *x_mu, const float *x_sd, const float *y_mu,
                          const float *y_sd);

/* Features of nq queries: d_seq (device) holds their ASCII letters back to
 * back, offsets (host, nq+1) delimit them; d_feat (device, nq x 66) receives
 * the features.  The index must be DNA. */
ae_status ae_mlp_features(const ae_index *idx, const uint8_t *d_seq, const int64_t *offsets, int32_t nq,
                          float *d_feat, void *stream);

/* Predictions for B feature rows: d_x (device, B x 66) -> d_y (device, B x 2),
 * in the units of the targets (log1p entries, log1p hits). */
ae_status ae_mlp_forward(ae_mlp *mlp, const float *d_x, int32_t B, float *d_y, void *stream);

/* Loss and gradient at the current parameters for B rows with targets d_t
 * (device, B x 2).  *loss (host) receives L; if grads (host, AE_MLP_PARAMS)
 * is not NULL it receives dL/dparams in the packed order.  No update. */
ae_status ae_mlp_loss_grad(ae_mlp *mlp, const float *d_x, const float *d_t, int32_t B, float *loss,
                           float *grads, void *stream);

/* Train on n rows (d_x: n x 66, d_t: n x 2, device) for `epochs` passes of
 * mini-batches of `batch` rows in an order shuffled per epoch from `seed`
 * (one Adam step of rate lr and weight decay weight_decay >= 0 per
 * mini-batch).  *loss (host, may be NULL) receives the mean mini-batch loss
 * of the last epoch. */
ae_status ae_mlp_train(ae_mlp *mlp, const float *d_x, const float *d_t, int32_t n, int32_t epochs,
                       int32_t batch, float lr, float weight_decay, uint64_t seed, float *loss, void *stream);

#ifdef __cplusplus
}
#endif

#endif
