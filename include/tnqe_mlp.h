/*
 * tnqe_mlp.h -- C ABI of the rotation-proposal network of the generalized
 * sweep: a fully connected network n_in -> n_hidden -> n_hidden -> n_out with
 * exact GELU activations, FP32, trained and evaluated on the GPU by this
 * library's own kernels (sm_103a).  The paper has no learned component; this
 * network proposes the orbital-rotation generator K of the next state in the
 * sweep of Sec. II C / App. A (its plain random proposal stays the fallback).
 *
 * Parameters, in this order, row-major FP32:
 *   W1 [n_hidden][n_in], b1 [n_hidden], W2 [n_hidden][n_hidden], b2 [n_hidden],
 *   W3 [n_out][n_hidden], b3 [n_out]
 * Forward:  Z1 = X W1^T + b1, A1 = gelu(Z1), Z2 = A1 W2^T + b2, A2 = gelu(Z2),
 *           Y = A2 W3^T + b3,  gelu(z) = z (1 + erf(z / sqrt 2)) / 2.
 * Loss (weighted mean squared error over a batch of B rows):
 *           L = sum_b w_b sum_o (Y_bo - T_bo)^2 / (n_out sum_b w_b).
 *
 * All arrays passed in are host memory and are copied; the caller keeps
 * ownership.  Every call returns a tnqe_status (include/tnqe.h); no exception
 * crosses the ABI.  One network per host thread.
 */
#ifndef TNQE_MLP_H
#define TNQE_MLP_H

#include "tnqe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnqe_mlp tnqe_mlp;

/* Create a network with zero parameters and zero Adam moments.  Sizes must be
 * in [1, 4096]; max_batch in [1, 65536] bounds every later batch.  stream: a
 * cudaStream_t, NULL = a stream owned by the network. */
tnqe_status tnqe_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, void* stream, tnqe_mlp** out);

/* Number of parameters (see the order above). */
long long tnqe_mlp_param_count(const tnqe_mlp* net);

/* Copy all parameters in / out (host arrays of tnqe_mlp_param_count floats).
 * set_params also clears the Adam moments and step count. */
tnqe_status tnqe_mlp_set_params(tnqe_mlp* net, const float* params);
tnqe_status tnqe_mlp_get_params(const tnqe_mlp* net, float* params);

/* Y [batch][n_out] = network(X [batch][n_in]). */
tnqe_status tnqe_mlp_forward(tnqe_mlp* net, const float* X, int batch, float* Y);

/* Loss and its gradient with respect to every parameter (grad may be NULL;
 * otherwise tnqe_mlp_param_count floats, same order as the parameters).
 * T [batch][n_out] targets, w [batch] non-negative row weights (NULL = 1). */
tnqe_status tnqe_mlp_gradient(tnqe_mlp* net, const float* X, const float* T, const float* w, int batch,
                              float* loss, float* grad);

/* One Adam step (Kingma & Ba, arXiv 1412.6980) on the loss of this batch:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * *loss (may be NULL) gets the loss before the step. */
tnqe_status tnqe_mlp_adam_step(tnqe_mlp* net, const float* X, const float* T, const float* w, int batch, float lr,
                               float beta1, float beta2, float eps, float* loss);

/* Kernels launched by the last call of this network. */
int tnqe_mlp_last_launches(const tnqe_mlp* net);

const char* tnqe_mlp_last_error(const tnqe_mlp* net);
void tnqe_mlp_destroy(tnqe_mlp* net);

#ifdef __cplusplus
}
#endif
#endif /* TNQE_MLP_H */
