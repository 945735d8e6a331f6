/*
 * oci_nn.h -- C ABI of the learned initial guess / corrector for the OCI
 * iteration: a small 1-D convolutional network over cells that predicts each
 * time step's converged scalar-flux moments from the last two steps' moments,
 * the cross sections, the cell widths and the source.
 *
 * The paper (arXiv 2305.13555) has no learned component; this network is an
 * addition whose only role is to change iteration counts (the OCI iteration
 * always runs to the same tolerance, see oci_nn_attach in oci.h).
 *
 * Network (fixed): 5 convolution layers along the cell index, kernel width 5,
 * zero padding of 2 cells at the slab ends, channels 13 -> 32 -> 32 -> 32 ->
 * 32 -> 4, ReLU after layers 1-4.  Parameters: one flat FP32 array, per layer
 * W[co][ci][5] (row-major) then b[co]; oci_nn_param_count() elements.  The
 * kernels use the weights rounded to BF16 and accumulate in FP32;
 * activations are FP32.
 *
 * Input channels per cell j (array in[b][13][J], FP32), with the per-sample
 * scale S = max(rms over cells and moments of phi1, rms of qfeat):
 *   0-3   phi1_c / S                   (phi1 = moments of step n-1)
 *   4-7   (phi1_c - phi2_c) / S        (phi2 = moments of step n-2)
 *   8-11  stat[j][0..3]                (static cell features, see below)
 *   12    qfeat[j] / S
 * Output out[b][4][J]: (phi_n - phi1) / S; the prediction is
 * phi_hat = phi1 + S * out (oci_nn_predict).
 * Static features as used by the library: log10(sigma_t)/2, c = sigma_s/sigma_t,
 * log10(sigma_t dx), log10(sigma_t v dt) (arguments of log10 floored at 1e-30);
 * qfeat = v dt (Q_kL + Q_kR)/2.
 *
 * Conventions: every pointer is a DEVICE pointer unless noted; arrays are C
 * row-major; work is enqueued on `stream` (cudaStream_t, NULL = legacy) and the
 * calls do not synchronise unless they return a host value.  Return codes are
 * the OCI_* codes of oci.h (0 ok, 1 invalid argument, 3 CUDA error).
 * Workspace: caller-owned device memory of oci_nn_workspace_bytes(B, J) bytes;
 * calls that share a workspace must not overlap.
 */
#ifndef OCI_GB300_OCI_NN_H
#define OCI_GB300_OCI_NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of FP32 parameters of the network. */
int32_t oci_nn_param_count(void);

/* Workspace bytes for a batch of `batch` samples of `n_cells` cells
 * (activations of every layer, gradients, per-tile partial sums). */
size_t oci_nn_workspace_bytes(int32_t batch, int32_t n_cells);

/* Build the input channels: phi1, phi2 [B][J][4] double; stat [B][J][4] and
 * qfeat [B][J] float; writes in [B][13][J] and the per-sample scale [B]. */
int oci_nn_features(const double *phi1, const double *phi2, const float *stat, const float *qfeat,
                    int32_t batch, int32_t n_cells, float *in, float *scale, void *stream);

/* Training targets (phi_n - phi1) / S: phin, phi1 [B][J][4] double,
 * scale [B] -> tgt [B][4][J]. */
int oci_nn_targets(const double *phin, const double *phi1, const float *scale, int32_t batch,
                   int32_t n_cells, float *tgt, void *stream);

/* Inference: in [B][13][J] -> out [B][4][J] with parameters params [count]. */
int oci_nn_forward(const float *params, const float *in, int32_t batch, int32_t n_cells, float *out,
                   void *workspace, size_t workspace_bytes, void *stream);

/* phi_hat = phi1 + S * out -> phat [B][J][4] double. */
int oci_nn_predict(const double *phi1, const float *out, const float *scale, int32_t batch,
                   int32_t n_cells, double *phat, void *stream);

/* Mean-squared-error loss over all outputs and its gradient with respect to
 * the (BF16-rounded) parameters: grad [count] (device, may be NULL), loss
 * (HOST pointer, may be NULL; if given the call synchronises `stream`). */
int oci_nn_loss_grad(const float *params, const float *in, const float *tgt, int32_t batch,
                     int32_t n_cells, float *grad, double *loss, void *workspace, size_t workspace_bytes,
                     void *stream);

/* One training step: loss and gradient as above, then Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected with step number `step` >= 1) on the
 * FP32 master parameters and moments adam_m, adam_v [count] (device, zeroed
 * before step 1).  loss: HOST pointer or NULL. */
int oci_nn_train_step(float *params, float *adam_m, float *adam_v, int32_t step, float lr, const float *in,
                      const float *tgt, int32_t batch, int32_t n_cells, double *loss, void *workspace,
                      size_t workspace_bytes, void *stream);

/* Largest n_cells accepted by oci_nn_forward_noalloc. */
#define OCI_NN_NOALLOC_MAX_CELLS 16384

/* Inference without any allocation (the paper has no counterpart): same
 * network, inputs and outputs as oci_nn_forward for a single sample (batch 1)
 * of at most OCI_NN_NOALLOC_MAX_CELLS cells, but the scratch memory (BF16
 * weights and two activation buffers, about 4.2 MB) is a fixed array inside
 * this library instead of a caller-provided workspace.  For callers that
 * cannot call cudaMalloc or pass scratch memory: code running where an
 * allocation would synchronise the device or is forbidden (a real-time step
 * loop, an inference hook inside another program's time step that owns the
 * memory plan), or a host that only hands over its input and output buffers.
 * Every GPU that loads the library holds the array until the process exits.
 * The first call on a device looks up the array's device address (with that
 * device current), so make the first call before any stream capture.  All
 * calls share the one array and it keeps the last call's contents: calls that
 * can overlap on the GPU (different streams, concurrent host threads) race,
 * so serialise them.  Nothing in it needs to start at zero.  in [13][n_cells]
 * and out [4][n_cells] are device pointers, params [oci_nn_param_count()].
 * Calls no cudaMalloc / cudaFree or allocating library routine.  Returns
 * 1 (OCI_EINVAL) for NULL pointers, n_cells < 1 or n_cells >
 * OCI_NN_NOALLOC_MAX_CELLS, 3 (OCI_ECUDA) on a CUDA error. */
int oci_nn_forward_noalloc(const float *params, const float *in, int32_t n_cells, float *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OCI_GB300_OCI_NN_H */
