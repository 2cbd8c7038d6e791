/*
 * Warm-start network of the dose engine: C ABI.
 *
 * The paper's Discussion ("Future directions") proposes a network that learns
 * delivery parameters from target and organ-at-risk masks, with the dose
 * engine judging its output.  This library implements such a proposal
 * network and its training on the GPU:
 *
 *   input   x   [n][64][64][3] BF16 (NHWC): beam's-eye-view projections of the
 *               PTV, bladder and rectum masks for one control point each
 *               (pdrt_bev_project);
 *   layers      four 3x3 stride-2 convolutions (zero padding 1, 64 channels,
 *               bias, ReLU; 64 -> 32 -> 16 -> 8 -> 4 pixels) and a dense head
 *               1024 -> 121 (bias, no activation);
 *   output  y   [n][121] FP32: 60 leaf pairs (left, right) then MU, in the
 *               normalised units the caller trains with.
 *
 * Weights and stored activations are BF16, every contraction accumulates in
 * FP32 (tcgen05 tensor cores); the FP32 master weights and the Adam state stay
 * on the device.  Parameter vector layout (FP32, pdrt_cnn_param_count floats):
 *   W1 [64][3][3][3], b1 [64], W2 [64][3][3][64], b2 [64], W3, b3, W4, b4
 *   (as W2, b2), W5 [121][1024] (input index (y*4 + x)*64 + c), b5 [121].
 *
 * All calls are asynchronous on `stream` unless stated; errors return a
 * pdrt_status and leave a message for pdrt_last_error (pdrt.h).  Handles are
 * not thread-safe; one stream per handle at a time.
 */
#ifndef PDRT_CNN_H
#define PDRT_CNN_H

#include "pdrt.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PDRT_CNN_SIDE 64     /* input pixels per side */
#define PDRT_CNN_IN_CH 3     /* PTV, bladder, rectum */
#define PDRT_CNN_OUT 121     /* 60 leaf pairs x 2 + MU */

typedef struct pdrt_cnn_s *pdrt_cnn_t;

/* Number of FP32 parameters (host-only). */
int64_t pdrt_cnn_param_count(void);

/* Creates a network for batches of up to batch_max samples; allocates all its
 * device memory (weights, Adam state, activations, gradients, split-K
 * partials) now.  Parameters start at zero: call pdrt_cnn_set_params.
 * Errors: EINVAL (batch_max < 1 or > 65536), ENOMEM, EDEVICE (not sm_103). */
pdrt_status pdrt_cnn_create(pdrt_cnn_t *out, int32_t batch_max, pdrt_stream_t stream);
void pdrt_cnn_destroy(pdrt_cnn_t net);

/* Copies the FP32 parameter vector from device memory (params_dev, caller
 * owned, pdrt_cnn_param_count floats) and resets the Adam state and step.
 * Errors (here and in every call below that takes a handle): EINVAL (NULL
 * handle or buffer, or the current device is not the handle's), ECUDA. */
pdrt_status pdrt_cnn_set_params(pdrt_cnn_t net, const float *params_dev, pdrt_stream_t stream);
/* Copies the FP32 master parameters to params_dev (caller owned). */
pdrt_status pdrt_cnn_get_params(pdrt_cnn_t net, float *params_dev, pdrt_stream_t stream);

/* Forward pass of n <= batch_max samples.  x_dev: BF16 bits [n][64][64][3];
 * y_dev: FP32 [n][121] (caller owned, overwritten).  The activations stay in
 * the handle for a following pdrt_cnn_backward of the same n.
 * Errors: ESHAPE (n outside 1..batch_max). */
pdrt_status pdrt_cnn_forward(pdrt_cnn_t net, const uint16_t *x_dev, int32_t n, float *y_dev,
                             pdrt_stream_t stream);

/* Backward pass of the last forward for an upstream gradient dy_dev FP32
 * [n][121] (rounded to BF16 like every backward operand); writes the FP32
 * parameter gradient to grads_dev (pdrt_cnn_param_count floats, caller owned)
 * or, if grads_dev is NULL, keeps it in the handle only.
 * Errors: ESHAPE (n is not the last forward's batch). */
pdrt_status pdrt_cnn_backward(pdrt_cnn_t net, int32_t n, const float *dy_dev, float *grads_dev,
                              pdrt_stream_t stream);

/* One training step: forward, mean-squared error against target_dev FP32
 * [n][121], backward and an Adam update (beta1 0.9, beta2 0.999, eps 1e-8)
 * with learning rate lr.  loss_dev (1 FP32, caller owned, may be NULL)
 * receives the batch loss before the update.
 * Errors: ESHAPE (n outside 1..batch_max), EINVAL (lr not positive and
 * finite). */
pdrt_status pdrt_cnn_train_step(pdrt_cnn_t net, const uint16_t *x_dev, const float *target_dev,
                                int32_t n, float lr, float *loss_dev, pdrt_stream_t stream);

/* Copies a buffer of the last forward of n samples to dst_dev (caller owned):
 * layer 0..4 = activations h_0..h_4 (BF16 NHWC, n * side^2 * channels
 * values), 5 = output (FP32 [n][121]).  Errors: EINVAL (layer), ESHAPE (n is
 * not the last forward's batch). */
pdrt_status pdrt_cnn_read_activation(pdrt_cnn_t net, int32_t layer, int32_t n, void *dst_dev,
                                     pdrt_stream_t stream);

/* Synchronises `stream`, returns and clears the device flags of the handle
 * (PDRT_FLAG_TIMEOUT if a tensor-core wait expired). */
pdrt_status pdrt_cnn_status(pdrt_cnn_t net, pdrt_stream_t stream, uint32_t *flags);

/*
 * Beam's-eye-view projection of structure masks (the network input).
 * masks_dev: uint8 [nz][ny][nx] (device), bit s set where the voxel belongs
 * to structure s (0 = PTV, 1 = bladder, 2 = rectum).  For control point b at
 * gantry angle gantry_deg[b] (host array) and BEV pixel (py, px) of a
 * side x side grid with pixel pitch pitch_mm at the isocentre plane
 * (u = (px - (side-1)/2) pitch along e_u = (cos g, -sin g, 0), v = (py -
 * (side-1)/2) pitch along e_v = +z), the ray from the source (at distance
 * sid_mm before the isocentre along e_w = (sin g, cos g, 0)) through
 * iso + u e_u + v e_v is sampled at depths -reach..+reach mm (step step_mm)
 * around the isocentre plane; channel s is 1 if a sample's nearest voxel has
 * bit s.  out_dev: BF16 bits [n_cp][side][side][3] (caller owned).
 * Geometry: voxel (i, j, k) centre at origin + (i sx, j sy, k sz) mm.
 * Errors: EINVAL (NULL, non-positive sizes, n_cp > 65535).
 */
pdrt_status pdrt_bev_project(const uint8_t *masks_dev, int32_t nx, int32_t ny, int32_t nz,
                             double sx, double sy, double sz, const double origin_mm[3],
                             const double iso_mm[3], double sid_mm, int32_t n_cp,
                             const double *gantry_deg, int32_t side, double pitch_mm,
                             double reach_mm, double step_mm, uint16_t *out_dev,
                             pdrt_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PDRT_CNN_H */
