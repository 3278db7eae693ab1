/*
 * asse_learn.h -- learned per-estimator cardinality model of the GB300 ASSE
 * library.  The paper has no learned component: Sec. 3 estimates an ATV's
 * cardinality with the linear-counting formula (Eq. 2), which saturates as
 * the ATV fills.  This model maps the state of one ATV to its log-cardinality
 * with a small MLP (features -> 256 -> 256 -> 1, ReLU), trained and run on the
 * GPU by the library's own BF16-in / FP32-accumulate kernels; Eq. 2 remains
 * the fallback outside the training range and the baseline it is compared with.
 *
 * Conventions as in asse.h (status codes, where = ASSE_HOST / ASSE_DEVICE,
 * stream-ordered asynchronous work unless stated).
 *
 * Feature row of one ATV (ASSE_FEAT bf16 values, the last 12 zero):
 *   [0]        |ATV|^{k'} / g            (active ATs, Algorithm 1)
 *   [1 + a]    (active ATs of age a) / g, a = 0..63, age = slices since the
 *              AT was set (a < k' <= 64)
 *   [65]       P = |AAT(k',i,j)| / (g 2^c), the load of the ATV's row i and
 *              frame j (Sec. 4.3)
 *   [66]       UP of its frame (product of P over the rows)
 *   [67]       mean of P over the rows of its frame
 * Target: ln(cardinality).
 */
#ifndef ASSE_LEARN_H
#define ASSE_LEARN_H

#include "asse.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ASSE_FEAT 80  /* feature row width */
#define ASSE_HID 256  /* hidden width */
/* parameters, in this order, as fp32: W1[HID][FEAT], b1[HID], W2[HID][HID],
 * b2[HID], w3[HID], b3 */
#define ASSE_MLP_NPARAMS (ASSE_HID * ASSE_FEAT + ASSE_HID + ASSE_HID * ASSE_HID + ASSE_HID + ASSE_HID + 1)

typedef struct asse_mlp asse_mlp;

/* Synthetic training states shaped like link-scale traffic: each state is
 * one ATV of g ATs over a window of k slices, holding one host of
 * cardinality n (log-uniform in [1, 2^n_max_log2], spread over the k slices
 * with random shares) plus background: every AT is independently set in each
 * slice with a probability p drawn uniformly in [0, bg_max] per state.  The
 * host's bips are distinct, so n is exact by construction. */
typedef struct asse_synth_cfg {
    uint32_t k, g, r;      /* window (<= 64), ATs per ATV, rows (for UP) */
    uint32_t n_max_log2;   /* cardinalities up to 2^n_max_log2 (<= 24) */
    float bg_max;          /* background probability range per AT and slice */
    uint32_t pad;
    uint64_t seed;         /* states are a pure function of (seed, index) */
    uint64_t bh_a, bh_b;   /* BH keys (bh_a odd), as in asse_config */
} asse_synth_cfg;

/* Feature rows of every ATV of a pool ([r*E][ASSE_FEAT] bf16 as uint16, in
 * ATV order), for the window and loads of the last asse_scan.  Valid between
 * asse_scan and asse_advance (the refresh changes the state).  Requires
 * kp <= 64.  Errors: ESTATE, EINVAL, ECUDA. */
ASSE_API int asse_features(asse_pool *pool, uint16_t *x_dev);

/* Learned cardinality estimate of every ATV of a pool, for the window of
 * the last asse_scan: the feature rows (written to x_dev, [r*E][ASSE_FEAT]
 * bf16, 16-byte aligned), the model on them, and est_dev[i] =
 * exp(max(model, 0)) where the ATV holds an active AT and the model is
 * inside its training range (model <= max_log_n, the log of the largest
 * cardinality it was trained on; a host has at least one bip), else Eq. 2's
 * linear-counting estimate from the ATV's count (0 for an empty ATV, a
 * saturated count g taken as g - 1/2).  *n_fallback_dev (device) receives
 * the number of ATVs that fell back to Eq. 2.  The model must run on the
 * pool's stream.  Same validity window as asse_features.
 * Errors: ESTATE, EINVAL, ECUDA. */
ASSE_API int asse_estimate_learned(asse_pool *pool, asse_mlp *mlp, float max_log_n, uint16_t *x_dev,
                                   float *est_dev, uint32_t *n_fallback_dev);

/* States first .. first+n-1 of a synthetic set: features x_dev [n][FEAT]
 * bf16, labels log_n_dev [n] = ln(n) and the Eq. 2 estimate of each state's
 * count lc_dev [n] (a saturated count g is taken as g - 1/2).  All device
 * buffers; stream-ordered on stream.  Errors: EINVAL, ECUDA. */
ASSE_API int asse_synth_states(const asse_synth_cfg *cfg, uint64_t first, uint64_t n, uint16_t *x_dev,
                               float *log_n_dev, float *lc_dev, void *stream);

/* Learned estimate of a candidate super point, in place of Eq. 4 (Sec. 4.3):
 * the same MLP (a separate instance) fed a feature row of the candidate
 * host built from its r ATVs instead of one ATV:
 *   [0]        NAT / g, the ATs active in all r ATVs (Algorithm 5)
 *   [1 + a]    ATs active in all r ATVs whose oldest timestamp over the rows
 *              is a slices old, / g (a < k' <= 64): the host sets all r ATs
 *              of a bip in the same slice, other hosts only make some younger
 *   [65]       UP of the host's frame (the product of the row loads, Eq. 4)
 *   [66], [67] the smallest and the largest row load P_i
 *   [68 + i]   |ATV_i|^{k'} / g of the host's ATV in row i (r <= 8)
 * Target: ln(cardinality). */

/* Candidate feature rows of n hosts (aips_dev, device) of a pool, for the
 * window and loads of the last asse_scan, into x_dev ([n][ASSE_FEAT] bf16,
 * device).  Same validity window as asse_features.
 * Errors: ESTATE, EINVAL, ECUDA. */
ASSE_API int asse_candidate_features(asse_pool *pool, const uint32_t *aips_dev, uint64_t n, uint16_t *x_dev);

/* The report of the last restore with the learned candidate estimate in
 * place of Eq. 4 (Sec. 4.3, Algorithm 5 and Eq. 4 decide the report of
 * asse_report; this build's model replaces that last step).  For every
 * candidate of CSIP (Algorithm 4): its feature row (as
 * asse_candidate_features), the model mlp on it (tensor-core inference),
 * and, where the model's output y is within its training range
 * (y <= max_log_n), est = exp(max(y, 0)) with flags ASSE_SP_LEARNED, and
 * ASSE_SP_REPORTED if est >= theta in FP32; elsewhere the candidate keeps its
 * Eq. 4 estimate, flags and decision.  The reported candidates are written
 * to out (host or device, `where`) in unspecified order, min(count, cap) of
 * them, and *n_out receives the count.  Every step runs on the device; the
 * call synchronises the pool's stream (it reads the candidate count first).
 * Valid between asse_scan + asse_restore and asse_advance, as
 * asse_features (after asse_close_slice the refresh has changed the
 * state: ESTATE).  The model must use the pool's stream.  The library keeps
 * the device workspace (about 200 bytes per candidate of the pool's list
 * capacity) with the model, allocated on first use.
 * Errors: EINVAL (NULL, negative max_log_n, other stream, k' > 64),
 * ESTATE, ECAPACITY (cap < count, *n_out set; or the restore overflowed, as
 * asse_report), ENOMEM, ETIMEOUT, ECUDA. */
ASSE_API int asse_report_learned(asse_pool *pool, asse_mlp *mlp, float max_log_n, asse_superpoint *out,
                                 uint64_t cap, uint64_t *n_out, int where);

/* Synthetic candidate states first .. first+n-1: one host of cardinality n
 * (log-uniform in [1, 2^n_max_log2], spread over the k slices with random
 * shares) in r ATVs, each row with its own background (every AT set in each
 * slice with a probability p_i drawn in [0, bg_max] per state and row); the
 * row loads are P_i = 1 - (1 - p_i)^k.  Outputs (device): feature rows x_dev
 * [n][ASSE_FEAT] bf16, log_n_dev [n] = ln(n), and eq4_dev [n], Eq. 4's
 * estimate from the state's NAT and UP (+inf when saturated).  cfg->r <= 8.
 * Stream-ordered on stream.  Errors: EINVAL, ECUDA. */
ASSE_API int asse_synth_candidates(const asse_synth_cfg *cfg, uint64_t first, uint64_t n, uint16_t *x_dev,
                                   float *log_n_dev, float *eq4_dev, void *stream);

/* A model with Kaiming-uniform weights drawn from seed and zero biases. */
ASSE_API int asse_mlp_create(uint64_t seed, void *stream, asse_mlp **out);
ASSE_API void asse_mlp_destroy(asse_mlp *mlp);
ASSE_API int asse_mlp_set_stream(asse_mlp *mlp, void *stream);

/* Copy all ASSE_MLP_NPARAMS fp32 parameters to / from host memory
 * (synchronises). */
ASSE_API int asse_mlp_get_params(asse_mlp *mlp, float *host);
ASSE_API int asse_mlp_set_params(asse_mlp *mlp, const float *host);

/* y_dev[i] = model(x_dev[i]) for n feature rows (device buffers; x_dev
 * 16-byte aligned, row-major [n][ASSE_FEAT]).  Inference runs the whole
 * network in one tensor-core kernel (tcgen05, accumulators in tensor memory,
 * BF16 operands, FP32 accumulation; H1 and H2 rounded to BF16 as in
 * training).  Stream-ordered; asse_mlp_check reports a kernel that failed.
 * Errors: EINVAL (misaligned x_dev), ECUDA. */
ASSE_API int asse_mlp_forward(asse_mlp *mlp, const uint16_t *x_dev, uint64_t n, float *y_dev);

/* Synchronise the model's stream; ASSE_ETIMEOUT if a kernel of this model
 * gave up a bounded wait (its outputs are then invalid), ASSE_ECUDA if a CUDA
 * call failed. */
ASSE_API int asse_mlp_check(asse_mlp *mlp);

/* Training losses over n rows with targets t_i = ln(cardinality):
 *   ASSE_LOSS_LOG_MSE  (1/n) sum (model(x_i) - t_i)^2, the squared error of
 *                      the log-estimate (default);
 *   ASSE_LOSS_REL_MSE  (1/n) sum (exp(model(x_i) - t_i) - 1)^2, the squared
 *                      relative error of the estimate exp(model) (model - t
 *                      clamped at 20), which favours the estimate with the
 *                      lowest relative error where a state says little
 *                      about its cardinality (a saturated estimator). */
#define ASSE_LOSS_LOG_MSE 0
#define ASSE_LOSS_REL_MSE 1

/* Select the loss of later asse_mlp_backward / asse_mlp_train_step calls.
 * Errors: EINVAL. */
ASSE_API int asse_mlp_set_loss(asse_mlp *mlp, int kind);

/* Gradients of the selected loss with respect to every parameter, for n rows
 * (device buffers); loss_dev (may be NULL) receives the loss.  Does not
 * change the parameters. */
ASSE_API int asse_mlp_backward(asse_mlp *mlp, const uint16_t *x_dev, const float *t_dev, uint64_t n,
                               float *loss_dev);

/* Copy the gradients of the last backward / train step to host memory
 * (ASSE_MLP_NPARAMS fp32, parameter order; synchronises). */
ASSE_API int asse_mlp_get_grads(asse_mlp *mlp, float *host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the gradients of n rows: backward then update. */
ASSE_API int asse_mlp_train_step(asse_mlp *mlp, const uint16_t *x_dev, const float *t_dev, uint64_t n, float lr,
                                 float *loss_dev);

/* Message of the last failing call on mlp. */
ASSE_API const char *asse_mlp_last_error(const asse_mlp *mlp);

#ifdef __cplusplus
}
#endif
#endif /* ASSE_LEARN_H */
