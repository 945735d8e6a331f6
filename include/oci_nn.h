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
 * kernels use the weights rounded to BF16 and accumulate in FP32.  Inference
 * (oci_nn_forward, oci_nn_forward_noalloc, the guess in oci_step) runs each
 * layer as a GEMM on the BF16 tensor cores, its input rounded to BF16
 * (oci_nn_forward and the guess: the five layers in one kernel, activations
 * in shared memory; oci_nn_forward_noalloc: one kernel per layer, the same
 * results bit for bit); training (oci_nn_loss_grad, oci_nn_train_step,
 * oci_nn_train) keeps the activations in FP32.
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
 * qfeat [B][J] float; writes in [B][13][J] and the per-sample scale [B].  The
 * scale's partial sums pass through `in` before the channels are written, so
 * `in` must not overlap the inputs. */
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

/* Trajectory data and controls of oci_nn_train. */
typedef struct {
    int32_t n_traj;            /* trajectories T >= 1 */
    int32_t n_steps;           /* steps S >= 1 per trajectory; sample (t, n), n = 1..S, predicts step n */
    int32_t n_cells;           /* cells J >= 1 (every trajectory the same size) */
    const double *phi;         /* [T][S+1][J][4]: moments of the initial state (n = 0) and of
                                  each converged step, as published by oci_fluxes_device */
    const float *stat;         /* [T][J][4] static features (oci_nn_static_features) */
    const float *qfeat;        /* [T][J] source feature (oci_nn_static_features) */
    int32_t epochs;            /* >= 1 */
    int32_t batch;             /* samples per minibatch, >= 1; the last incomplete batch of an
                                  epoch is dropped */
    float lr;                  /* peak learning rate; epoch e (0-based) uses
                                  lr (1 + cos(pi e / epochs)) / 2 */
    float val_frac;            /* fraction of the samples held out for validation, in [0, 1) */
    uint64_t seed;             /* shuffle (and, with init_params NULL, initialisation) seed */
    const float *init_params;  /* [count] starting parameters, or NULL for the library's
                                  initialisation (below) */
    void *stream;              /* cudaStream_t for all work */
} oci_nn_train_cfg;

/* What oci_nn_train did (host struct). */
typedef struct {
    int32_t epochs_done, steps_done;  /* Adam steps taken (step numbers 1..steps_done) */
    int32_t n_train, n_val;           /* samples in the training and validation sets */
    double train_loss;                /* mean loss of the sampled minibatches of the last epoch
                                         (every 50th minibatch, starting with the first) */
    double val_loss;                  /* mean loss over the validation minibatches after the last
                                         epoch (batches of min(batch, n_val) samples; NaN if n_val = 0) */
} oci_nn_train_stats;

/* The whole training procedure of the network on trajectories that the
 * library's own solver produced (the paper has no counterpart): minibatch
 * Adam (oci_nn_train_step) on the mean-squared error of oci_nn_targets, with
 * the sample order, the train/validation split and the learning-rate
 * schedule fixed here so that a run is reproducible bit for bit.
 *   Samples are numbered k = t S + (n - 1).  Shuffles are Fisher-Yates passes
 *   "for i = len-1 down to 1: swap a[i] and a[j], j = h mod (i + 1)" with
 *   h = splitmix64(seed + r * 2^32 + i), splitmix64 being Vigna's finaliser
 *   (z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
 *   z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31), all modulo 2^64.
 *   Round r = 0 shuffles the list 0..T S - 1; its first floor(T S val_frac)
 *   entries are the validation set, the rest the training list, which round
 *   r = e + 1 shuffles in place at the start of epoch e.  Minibatch b of an
 *   epoch is training-list entries [b batch, (b + 1) batch); Adam step numbers
 *   count from 1 over the whole run.
 *   Initialisation when init_params is NULL: every weight of a layer with CI
 *   input channels is sqrt(6 / (5 CI)) (2 u - 1), u = (splitmix64(seed ^
 *   0x5DEECE66D + i) >> 11) 2^-53 for flat parameter index i; biases 0.
 * weights_out: DEVICE [count], the trained FP32 parameters.  stats: HOST, may
 * be NULL.  Allocates its own device buffers (released before it returns) and
 * synchronises `stream` while it runs.  Returns 0, 1 (OCI_EINVAL) for NULL
 * data or out-of-range sizes, 2 (OCI_ENOMEM), 3 (OCI_ECUDA). */
int oci_nn_train(const oci_nn_train_cfg *cfg, float *weights_out, oci_nn_train_stats *stats);

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
 * device current), so make the first call before any stream capture; after a
 * reset of the device's primary context (cudaDeviceReset) the next call looks
 * it up again, so make that call before any capture too.  Devices with an
 * index of 64 or more are not supported (OCI_EINVAL).  All
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
