/*
 * ranc_mlp.h - C ABI of the design-space surrogate: a small fully connected
 * network (ReLU hidden layers, linear output) trained on simulator outputs to
 * rank candidate RANC configurations, so that only the best-ranked ones are
 * simulated exactly.  The paper motivates fast design-space exploration over
 * RANC's many configuration parameters (Sec. I and Sec. V: numbers and bit
 * widths of weights, axons and neurons per core, leak and threshold values)
 * but trains no model; this is the project's own component.
 *
 * Numerics: weights are held as bf16 for the forward and backward passes, with
 * fp32 master copies updated by Adam; activations and gradients are fp32.
 * Every matrix product runs on the tensor cores (mma.sync bf16 -> fp32
 * accumulation): a bf16 weight enters exactly, an fp32 activation or gradient
 * as two bf16 terms hi + lo (16 significant bits), and a product of two fp32
 * operands as hi*hi + hi*lo + lo*hi.  The loss is the mean squared error over
 * the batch and the outputs.
 *
 * Conventions as in ranc.h: 0 or a negative RANC_E* code, reason in
 * ranc_mlp_last_error; all work on the stream given at creation; "device"
 * pointers are caller-owned CUDA memory; the handle owns its parameters,
 * optimizer state and activation buffers.  Not thread-safe per handle.
 */
#ifndef RANC_MLP_H
#define RANC_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ranc_mlp ranc_mlp;

/* n_layers >= 1 linear layers; dims[0] inputs, dims[n_layers] outputs, every
 * dim in [1, 1024]; max_batch >= 1 rows per call.  Weights are initialised
 * from `seed` (uniform in +-sqrt(6 / fan_in)), biases to zero. */
int ranc_mlp_create(int32_t n_layers, const int32_t *dims, int32_t max_batch, uint64_t seed, void *cuda_stream,
                    ranc_mlp **out);

/* Number of parameters: sum over layers of dims[l+1] * dims[l] + dims[l+1]. */
int ranc_mlp_param_count(const ranc_mlp *m, int64_t *count);

/* Host copies of the parameters in layer order, each layer's weight matrix
 * [dims[l+1]][dims[l]] (row major) then its bias.  ranc_mlp_get_params returns
 * the bf16-rounded weights the passes use (as floats); ranc_mlp_set_params sets
 * the fp32 masters (and their bf16 copies) and clears the optimizer state.
 * Synchronous. */
int ranc_mlp_get_params(ranc_mlp *m, float *params);
int ranc_mlp_set_params(ranc_mlp *m, const float *params);

/* y [batch][dims[n_layers]] = network(x [batch][dims[0]]), device pointers,
 * batch <= max_batch.  Stream-ordered. */
int ranc_mlp_forward(ranc_mlp *m, const float *x, int32_t batch, float *y);

/* Forward, MSE loss against target [batch][dims[n_layers]] and backward pass
 * into the handle's gradient buffers (device pointers in, loss out to host).
 * grads, when not NULL, receives the gradients in the layout of
 * ranc_mlp_get_params (host).  Synchronous when loss or grads is requested. */
int ranc_mlp_loss_backward(ranc_mlp *m, const float *x, const float *target, int32_t batch, float *loss,
                           float *grads);

/* One Adam step (bias-corrected) on the fp32 masters from the last
 * ranc_mlp_loss_backward, then refresh of the bf16 weights.  Stream-ordered. */
int ranc_mlp_adam_step(ranc_mlp *m, float lr, float beta1, float beta2, float eps);

void ranc_mlp_destroy(ranc_mlp *m);
const char *ranc_mlp_last_error(const ranc_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* RANC_MLP_H */
