/*
 * dvnr.h -- C ABI of libdvnr.so, the GB300 (sm_103a) implementation of the
 * hot path of "Distributed Neural Representation for Reactive In Situ
 * Visualization" (DVNR, arXiv 2304.10516).
 *
 * The library trains one implicit neural representation (INR) per box
 * partition of a volume (Sec. 3.1), with no exchange between partitions, and
 * decodes and ray-marches the trained models (Sec. 3, Sec. 4.3). Each INR is
 * a multiresolution hash-grid encoding (Sec. 3, after Mueller et al. 2022)
 * followed by a small ReLU MLP without biases and with a linear scalar
 * output (Sec. 3).
 *
 * Conventions shared by every call:
 *  - Device pointers ("_dev") point to memory of the current CUDA device;
 *    the caller owns them. The library owns model parameters, optimiser
 *    state and workspaces. Volumes are only borrowed during dvnr_train
 *    (the paper revokes field access after training, Sec. 4.1).
 *  - Volumes are float32, x fastest, then y, then z ([z][y][x]).
 *  - "stream" is a cudaStream_t (NULL = legacy default stream). Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Every call returns a dvnr_status; nothing aborts or traps. On an error
 *    dvnr_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread). Argument errors are detected on the host before
 *    any work is queued. Errors found by kernels (non-finite input, a
 *    non-finite gradient) are recorded in the model's device state and
 *    reported by the next synchronising call (dvnr_get_state, or dvnr_train
 *    with final_loss_host != NULL).
 *  - The library is compute-only: it uses one GPU and no collectives.
 *
 * Fixed-point coordinates: the INR domain of a model is [0,1]^3 spanning the
 * centres of the first and last stored voxel (ghost layer included). A unit
 * coordinate u is represented exactly as m / 2^24 with the integer
 * m in [0, 2^24]; hash indices and trilinear weights are computed from m.
 */
#ifndef DVNR_H
#define DVNR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DVNR_ABI_VERSION 1

typedef struct dvnr_model_s* dvnr_model; /* opaque, library-owned */

typedef enum {
  DVNR_OK = 0,
  DVNR_E_INVALID = 1,          /* bad argument (host-side check)            */
  DVNR_E_OOM = 2,              /* device allocation failed                  */
  DVNR_E_CUDA = 3,             /* a CUDA runtime call failed                */
  DVNR_E_NONFINITE_INPUT = 4,  /* NaN/Inf found in a training volume        */
  DVNR_E_TIMEOUT = 5,          /* a bounded device wait gave up             */
  DVNR_E_STATE = 6,            /* call not valid in the model's state       */
  DVNR_E_UNSUPPORTED = 7       /* configuration outside the compiled set    */
} dvnr_status;

typedef enum { DVNR_FP32 = 0, DVNR_FP16 = 1 } dvnr_precision;
typedef enum { DVNR_LOSS_L1 = 0, DVNR_LOSS_L2 = 1 } dvnr_loss;

/* Partition box in global voxel indices (Sec. 3.1: each rank owns a box).
 * Owned voxels are [lo, hi) per axis; the stored block adds `ghost` layers
 * on every side (Sec. 3.3, one ghost layer), so it has
 * (hi - lo + 2 ghost) voxels per axis, at least 2.                          */
typedef struct {
  int64_t lo[3], hi[3];
  int32_t ghost;
} dvnr_box;

/* Hash-grid encoding (Sec. 3, appendix network configs: n_levels,
 * n_features_per_level, log2_hashmap_size, base_resolution,
 * per_level_scale). Level l has resolution N_l = floor(base_res growth^l);
 * it is stored densely when (N_l+1)^3 <= 2^log2_T, else hashed into 2^log2_T
 * entries with the spatial hash of Mueller et al.
 * Supported: 1 <= n_levels <= 32, n_features in {1,2,4,8},
 * 4 <= log2_T <= 24, N_l <= 2^21.                                           */
typedef struct {
  int32_t n_levels, n_features, log2_T, base_res;
  double growth;
} dvnr_enc_cfg;

/* ReLU MLP (Sec. 3; appendix: n_neurons, n_hidden_layers). n_hidden hidden
 * layers of `width` units, then one linear output. No biases.
 * Supported: width in {16, 32, 64}, 1 <= n_hidden <= 8. The FP16 path also
 * needs n_levels * n_features at most 64 and n_features in {1, 2, 4, 8}; an
 * encoding width that is not a multiple of 16 (the appendix's 5 levels x 4
 * features, for one) enters the first layer padded with zero features.     */
typedef struct {
  int32_t width, n_hidden;
} dvnr_mlp_cfg;

/* Training configuration (Sec. 3.2 batch, Sec. 3.3 lambda/sigma, Sec. 3.6
 * Adam beta1 = 0.9, beta2 = 0.999, eps = 1e-8, L2 weight decay 1e-9,
 * boundary weight lambda = 0.15, sigma = 0.005).
 *   batch          samples per model per step (N_batch), >= 1
 *   lambda_bnd     fraction of boundary samples, floor(lambda batch)
 *   sigma_bnd      half-Gaussian spread in unit coordinates, (0, 1]
 *   precision      DVNR_FP32: plain FP32 SIMT path, one model at a time
 *                  DVNR_FP16: FP16 tables and MLP operands on tcgen05
 *                  tensor cores, FP32 accumulation, FP32 master weights and
 *                  Adam, dynamic loss scaling; all models of the call that
 *                  share an encoding and MLP configuration in one grouped
 *                  launch per step (models with adaptive table sizes form
 *                  one group per configuration)
 *   loss           DVNR_LOSS_L1 (paper) or DVNR_LOSS_L2
 *   growth_interval  FP16 path: finite steps before the loss scale doubles
 *   steps          N_train: fixed iteration count of this call (>= 0),
 *                  used when epochs == 0
 *   seed           sampling seed; model i of the call uses RNG key
 *                  (seed, i) -- the Philox counter also carries the model's
 *                  iteration count, so repeated calls draw fresh samples.
 *   epochs         N_epoch (>= 0): when > 0 the iteration count of model i
 *                  is ceil(N_vox_i / batch) * epochs, N_vox_i = its owned
 *                  voxels (Sec. 3.2: iterations proportional to the voxel
 *                  count of the partition)
 *   min_steps      N_train^min (>= 0): every model's count is at least this,
 *                  so N_train^max = max(min_steps, count) (Sec. 3.2)
 *   stop_loss      early stop (Sec. 3.2): a model stops once the moving
 *                  average of its training loss falls below stop_loss
 *                  (0 = off, else > 0)
 *   stop_decay     the moving average: m_1 = L_1, m_t = d m_{t-1} +
 *                  (1 - d) L_t over the finite steps of this call,
 *                  d = stop_decay in [0, 1)
 * Models of one call keep their own budgets: a model that reached its
 * N_train^max or its stop threshold does no further work in the call (its
 * tiles leave the grouped launch) while the others go on.                    */
typedef struct {
  float lr, beta1, beta2, eps, weight_decay;
  float lambda_bnd, sigma_bnd;
  int32_t batch, precision, loss, growth_interval;
  int64_t steps;
  uint64_t seed;
  int64_t epochs, min_steps;
  float stop_loss, stop_decay;
} dvnr_train_cfg;

/* Snapshot of a model (read synchronously by dvnr_get_state).              */
typedef struct {
  double vmin, vmax;       /* value range of the last training volume (Sec. 4.1) */
  double loss_scale;       /* FP16 path dynamic loss scale                     */
  double last_loss;        /* mean loss of the last step                       */
  int64_t iter;            /* iterations drawn                                  */
  int64_t adam_t;          /* Adam steps applied                                */
  int64_t skipped;         /* steps skipped: non-finite gradient, or a step     */
                           /*   a bounded device wait aborted                   */
  int64_t n_enc, n_mlp;    /* parameter counts                                  */
  int32_t precision;       /* precision used by decode/render                   */
  int32_t nonfinite_input; /* 1 when the last training volume held NaN/Inf      */
  double loss_ema;         /* moving average of the loss in the last call       */
                           /*   (-1 before the first finite step)               */
  int64_t budget_end;      /* iteration at which the last call's budget ends    */
  int32_t stopped;         /* 1 when the last call stopped on stop_loss         */
  int32_t frozen;          /* 1 after dvnr_freeze                               */
} dvnr_state_info;

/* Transfer function for dvnr_render: rgb = c0 + (c1 - c0) v and
 * alpha = alpha_max v, with v = clamp((value - v_lo)/(v_hi - v_lo), 0, 1).  */
typedef struct {
  float c0[3], c1[3];
  float alpha_max, v_lo, v_hi;
} dvnr_tf;

/* Optional device outputs of dvnr_train_grad (each may be NULL).           */
typedef struct {
  float* grad;       /* n_enc + n_mlp: gradient of the mean loss (unscaled)  */
  float* y;          /* batch: network output in normalised units            */
  float* target;     /* batch: normalised target                              */
  float* dx0;        /* batch x (n_levels n_features): dL/d(encoding),        */
                     /*   unscaled, level-major                               */
  uint32_t* coords;  /* batch x 3: fixed-point sample coordinates             */
  float* loss;       /* 1: mean loss of the batch                             */
} dvnr_step_outputs;

/* ABI version (DVNR_ABI_VERSION of the built library).                     */
int32_t dvnr_abi_version(void);

/* Message of the last failed call on this thread ("" if none).             */
const char* dvnr_last_error(void);

/* Create one INR for the partition `box` (Sec. 3.1) on the current device.
 * Parameters are initialised from `seed` (tables U(-1e-4, 1e-4), MLP
 * Glorot-uniform; Philox-4x32-10 counter {i_lo, i_hi, 0, 'INIT'},
 * key = seed), Adam moments are zero, value range [0, 1], precision FP32.
 * Synchronises the device. Errors: DVNR_E_INVALID (box/config),
 * DVNR_E_UNSUPPORTED, DVNR_E_OOM, DVNR_E_CUDA.                              */
dvnr_status dvnr_create(const dvnr_box* box, const dvnr_enc_cfg* enc,
                        const dvnr_mlp_cfg* mlp, uint64_t seed,
                        dvnr_model* out);

/* Adaptive encoding of a partition (Sec. 3.2: the hash table size and the
 * base resolution follow the partition's share of the global voxel count,
 * keeping the total model size of a decomposition near T_ref):
 *   T   = max(2^log2_T_min, T_ref n_vox / n_vox_global rounded up to a power
 *         of two), T_ref = 2^log2_T_ref
 *   R_0 = floor(R_ref (T / T_ref)^(1/3)), at least 1
 * (the paper prints T = max(T_min, T_ref ceil(N_vox / N_vox^global)), whose
 * ceiling is 1 for every partition; the ceiling is read as applying to the
 * product). Sets enc->log2_T and enc->base_res and leaves the other fields.
 * Host arithmetic only (exact for integer R_ref). Errors: DVNR_E_INVALID
 * unless 1 <= n_vox <= n_vox_global, 1 <= log2_T_min <= log2_T_ref <= 31,
 * R_ref >= 1 and finite.                                                    */
dvnr_status dvnr_adaptive_encoding(int64_t n_vox, int64_t n_vox_global, int32_t log2_T_ref,
                                   int32_t log2_T_min, double R_ref, dvnr_enc_cfg* enc);

/* Free a model (NULL is ignored). Synchronises the model's device.         */
void dvnr_destroy(dvnr_model m);

/* Freeze a trained model for storage (Sec. 4.2 keeps trained models for
 * later access; Sec. 3.4 stores them as 16-bit floats): keep only its FP16
 * parameters and value range on the device (2 bytes per parameter plus
 * 256-byte-aligned state) and free the FP32 weights, the Adam moments, the
 * gradients and every workspace. A frozen model decodes, renders and
 * exports in FP16 and can warm-start another model (dvnr_copy_weights
 * widens its FP16 parameters); training it, setting or importing its
 * weights or switching it to FP32 returns DVNR_E_STATE. dvnr_get_weights
 * returns the widened FP16 parameters. Synchronises `stream`; freezing a
 * frozen model does nothing. Needs a configuration the FP16 path supports. */
dvnr_status dvnr_freeze(dvnr_model m, void* stream);

/* Parameter counts: tables (n_enc) and MLP weights (n_mlp).                */
dvnr_status dvnr_param_count(dvnr_model m, int64_t* n_enc, int64_t* n_mlp);

/* Copy the FP32 master parameters to/from host memory (n = n_enc + n_mlp
 * floats, layout: tables level by level, entries x features with features
 * contiguous; then W_0 [width x in_dim], W_1..W_{H-1} [width x width],
 * w_out [width], each row-major [out][in]). set_weights also refreshes the
 * FP16 copy and resets the optimiser state (moments, step counts, loss
 * scale). Both synchronise.                                                 */
dvnr_status dvnr_get_weights(dvnr_model m, float* host, int64_t n);
dvnr_status dvnr_set_weights(dvnr_model m, const float* host, int64_t n);

/* Model export as 16-bit floats (Sec. 3.4 stores the weights as 16-bit
 * floats): the FP16 copy of the parameters (binary16 round-to-nearest-even of
 * the FP32 master weights), n = n_enc + n_mlp values in the compact layout of
 * dvnr_get_weights, as IEEE binary16 bit patterns. Import sets the FP32
 * master weights to the widened FP16 values, refreshes the FP16 copy and
 * resets the optimiser state. Both synchronise.                             */
dvnr_status dvnr_export_fp16(dvnr_model m, uint16_t* host, int64_t n);
dvnr_status dvnr_import_fp16(dvnr_model m, const uint16_t* host, int64_t n);

/* Weight caching (Sec. 3.5): initialise `dst` from `src` (same encoding and
 * MLP configuration), copying parameters and value range and resetting
 * dst's Adam moments and step counts. Asynchronous on `stream`.            */
dvnr_status dvnr_copy_weights(dvnr_model dst, dvnr_model src, void* stream);

/* Select the precision used by decode and render (training sets it to the
 * training precision). Switching to FP16 refreshes the FP16 copy.          */
dvnr_status dvnr_set_precision(dvnr_model m, int32_t precision, void* stream);

/* Synchronous snapshot of the model state; reports DVNR_E_TIMEOUT if a
 * bounded device wait gave up since the start of the last training call (in
 * that call or in a decode after it), else DVNR_E_NONFINITE_INPUT if the last
 * training volume held NaN/Inf (the state is filled in either way).        */
dvnr_status dvnr_get_state(dvnr_model m, dvnr_state_info* out);

/* Set the value range that decoding de-normalises with (Sec. 4.1: outputs
 * are y (vmax - vmin) + vmin), as training sets it from its volume: for a
 * model restored from stored weights. vmin <= vmax, both finite (stored as
 * float32); else DVNR_E_INVALID. Allowed on frozen models. Ordered after the
 * work already on `stream`; synchronises the stream.                       */
dvnr_status dvnr_set_value_range(dvnr_model m, double vmin, double vmax, void* stream);

/* Train n models for cfg->steps iterations each (Sec. 3.2): per step and
 * model, sample cfg->batch coordinates (uniform and boundary, Sec. 3.3),
 * look up targets by trilinear interpolation of the model's volume after
 * min/max normalisation (Sec. 3.1), run the encoding and MLP forward, the
 * L1 (or L2) loss, the backward pass with the gradient scatter into the
 * tables, and one Adam step. vol_dev[i] is model i's stored block
 * ((hi-lo+2 ghost) voxels per axis). The value range is taken from the
 * volume first (min/max over all stored voxels).
 * FP16 precision: the models that share an encoding and MLP configuration
 * run in one grouped kernel per step (one such launch per configuration
 * present in the call), the steps are replayed from a CUDA graph. When the
 * models' budgets differ or cfg->stop_loss is set, a call's steps run as a
 * conditional WHILE graph node that ends once no model is active (the
 * budget and stop tests run on the device; the host reads nothing during
 * the call); a runtime that refuses conditional nodes, or the environment
 * variable DVNR_GRAPH_LOOP=0, gets a fixed graph whose steps do nothing for
 * models that left. The first FP16 call for a configuration (encoding, MLP,
 * batch, number of models) times a few launch shapes of the training kernel
 * on its models and volumes and keeps the fastest for the process; that call
 * synchronises the stream once (parameters, moments and step counters are
 * not changed by the trials; environment variable DVNR_AUTOTUNE=0 skips it).
 * FP32 precision: the plain path, models one after another.
 * final_loss_host: if not NULL, receives n mean losses of the last step
 * and the call synchronises the stream.
 * Errors: DVNR_E_INVALID, DVNR_E_UNSUPPORTED, DVNR_E_CUDA,
 * DVNR_E_NONFINITE_INPUT (only when synchronising).                         */
dvnr_status dvnr_train(dvnr_model* models, int32_t n,
                       const float* const* vol_dev, const dvnr_train_cfg* cfg,
                       void* stream, float* final_loss_host);

/* One training step's forward and backward without the optimiser: the
 * batch of iteration `iteration` (Philox counter), model slot 0, value range
 * taken from vol_dev. Writes the requested outputs (see dvnr_step_outputs);
 * the model's parameters and optimiser state are unchanged. Uses the same
 * kernels as dvnr_train for cfg->precision (the FP16 path at loss scale
 * 2^round(log2 batch)).                                                     */
dvnr_status dvnr_train_grad(dvnr_model m, const float* vol_dev,
                            const dvnr_train_cfg* cfg, int64_t iteration,
                            const dvnr_step_outputs* out, void* stream);

/* One Adam step (Sec. 3.6: beta1, beta2, eps, L2 weight decay added to the
 * gradient, Kingma & Ba bias correction) from a gradient the caller supplies
 * instead of one training step's: grad_dev holds n_enc + n_mlp float32 values
 * on the device in the compact layout of dvnr_get_weights, the gradient of the
 * loss (not loss-scaled). Uses cfg->lr, beta1, beta2, eps, weight_decay and
 * precision (and cfg->batch for the FP16 path's initial loss scale when the
 * model has none yet). The same fused optimiser kernel as dvnr_train: the FP32
 * master weights, both moments and the FP16 copy are updated and the gradient
 * buffer is cleared. FP16 precision: the gradient is multiplied by the loss
 * scale S before the step (Adam divides it out); a value that is or becomes
 * non-finite skips the step and halves S, and growth_interval finite steps
 * double it, as in training. FP32 precision: S = 1; a non-finite value skips
 * the step. The iteration count, the last loss and its moving average are
 * not changed. Asynchronous on `stream`. Errors: DVNR_E_INVALID,
 * DVNR_E_STATE (frozen model), DVNR_E_UNSUPPORTED, DVNR_E_CUDA.             */
dvnr_status dvnr_adam_step(dvnr_model m, const float* grad_dev, const dvnr_train_cfg* cfg,
                           void* stream);

/* Copy the Adam moments (first m1, second m2; FP32) to host memory in the
 * compact layout of dvnr_get_weights, n = n_enc + n_mlp each; either pointer
 * may be NULL. Synchronises the device. DVNR_E_STATE for a frozen model.    */
dvnr_status dvnr_get_moments(dvnr_model m, float* m1_host, float* m2_host, int64_t n);

/* The network as a differentiable function of its parameters (Sec. 3: the
 * INR is the hash-grid encoding followed by the MLP; Sec. 3.6: trained by
 * back-propagation through both), for callers that build their own losses
 * (e.g. a torch.autograd.Function). Coordinates are fixed point, as in
 * training: coords_dev holds n x 3 uint32 values m in [0, 2^24], u = m 2^-24
 * in the model's unit domain. precision selects the kernels: DVNR_FP32 the
 * plain FP32 path (FP32 master weights), DVNR_FP16 the tensor-core path
 * (the FP16 copy of the weights, the training kernel's rounding points).
 *
 * load_params: set the FP32 master weights from params_dev (n_enc + n_mlp
 *   float32 on the device, compact layout of dvnr_get_weights) and refresh
 *   the FP16 copy; Adam moments and step counters are kept. Asynchronous.
 * forward: y_dev[i] = network output at point i, in normalised units (no
 *   value range applied). Asynchronous.
 * backward: the gradient of L with respect to every parameter, given
 *   dy_dev[i] = dL/dy_i (n float32): grad_dev receives n_enc + n_mlp float32
 *   in the compact layout (tables, then the MLP weights), dx0_dev (may be
 *   NULL) the n x (n_levels n_features) values dL/d(encoding). The same
 *   fused training kernel as dvnr_train with the loss replaced by dy and the
 *   samples by the given points. FP16: dy is multiplied by a loss scale S
 *   before the backward pass and every gradient divided by it again:
 *   loss_scale > 0 is used as given, 0 picks S = 2^k with max|dy| S in
 *   [1, 2) (S = 1 when dy is zero or not finite); FP32 ignores loss_scale.
 *   Non-finite values propagate into the outputs. Uses the model's gradient
 *   buffer (zero between calls), so it must not overlap a training call of
 *   the same model. 1 <= n <= 2^30. Synchronises `stream`.
 * Errors: DVNR_E_INVALID, DVNR_E_STATE (frozen model; FP32 forward of a
 * frozen model), DVNR_E_UNSUPPORTED, DVNR_E_CUDA.                            */
dvnr_status dvnr_load_params(dvnr_model m, const float* params_dev, void* stream);
dvnr_status dvnr_forward(dvnr_model m, const uint32_t* coords_dev, int64_t n, int32_t precision,
                         float* y_dev, void* stream);
dvnr_status dvnr_backward(dvnr_model m, const uint32_t* coords_dev, int64_t n, const float* dy_dev,
                          int32_t precision, float loss_scale, float* grad_dev, float* dx0_dev,
                          void* stream);

/* Point inference (Sec. 3, Sec. 4.1): n points in global voxel coordinates
 * (x, y, z float32 triples; voxel centre of global index j is at j) mapped
 * into the model's unit domain, clamped to it, evaluated and de-normalised
 * with the stored value range: out = y (vmax - vmin) + vmin.              */
dvnr_status dvnr_decode_points(dvnr_model m, const float* xyz_dev, int64_t n,
                               float* out_dev, void* stream);

/* Decode to the grid (Sec. 3, Sec. 4.1): the owned voxels of the box,
 * (hi-lo) per axis, x fastest, float32.                                     */
dvnr_status dvnr_decode_grid(dvnr_model m, float* out_dev, void* stream);

/* Direct volume rendering of n models (Sec. 4.3, reading stated in the
 * project notes): each model is decoded to its owned grid, then one ray per
 * pixel is marched orthographically along +z through the union of the owned
 * boxes with spr samples at the centres of equal steps, trilinear on the
 * grid of the block that owns the sample (clamped at that block's edge),
 * transfer function `tf`, front-to-back compositing without early
 * termination (sort-last order along +z). rgba_dev: h x w x 4 float32,
 * premultiplied colour and opacity.                                         */
dvnr_status dvnr_render(const dvnr_model* models, int32_t n, const dvnr_tf* tf,
                        int32_t w, int32_t h, int32_t spr, float* rgba_dev,
                        void* stream);

/* Rendering in a given frame, for sort-last compositing (Sec. 4.3: every
 * rank renders its own partitions, the images are blended in depth order).
 * As dvnr_render (from_network = 0: decoded grids) or dvnr_render_inr
 * (from_network = 1: the networks), but the camera spans the box
 * [frame_lo, frame_hi) (global voxel indices, hi > lo per axis) instead of
 * the union of the models' boxes, so images of disjoint partition sets
 * rendered apart in one frame align pixel for pixel and sample for sample;
 * pixels whose ray misses the models are (0, 0, 0, 0).                     */
dvnr_status dvnr_render_in_frame(const dvnr_model* models, int32_t n, const int64_t frame_lo[3],
                                 const int64_t frame_hi[3], const dvnr_tf* tf, int32_t w,
                                 int32_t h, int32_t spr, int32_t from_network, float* rgba_dev,
                                 void* stream);

/* Sort-last compositing (Sec. 4.3): blend n premultiplied RGBA images of one
 * frame (w x h x 4 float32 on the device each) front to back in increasing
 * depth_host[i] (e.g. the lo.z of the partitions each was rendered from;
 * ties keep the input order): C += (1 - A) C_i, A += (1 - A) A_i. For
 * partitions whose boxes are disjoint and ordered along +z this gives the
 * image of their union (up to rounding order). out_dev may not alias an
 * input. Synchronises the stream.                                           */
dvnr_status dvnr_composite(const float* const* rgba_dev, const double* depth_host, int32_t n,
                           int32_t w, int32_t h, float* out_dev, void* stream);

/* Temporal sliding window of models (Sec. 4.2: the most recent time steps
 * stay available as trained models; when the window is full the oldest
 * step is dropped). A step holds one model per partition (n_parts boxes,
 * each with its own encoding, e.g. from dvnr_adaptive_encoding; one MLP).
 *  - push: creates the step's models, warm-starts them from the newest step
 *    (Sec. 3.5 weight caching: parameters and value range copied, Adam
 *    reset; the first step starts from `seed` + part), trains them on the
 *    n_parts volumes with dvnr_train(cfg), then drops the oldest step if
 *    the window held `capacity` steps and freezes the previous newest step
 *    (dvnr_freeze): only the newest step keeps trainable FP32 state.
 *    *t_out = the step's index (0, 1, ...); final_loss_host as dvnr_train.
 *    On an error the new step is discarded and the cached steps stay
 *    (a model whose freezing failed stays trainable).
 *  - range: indices of the oldest and newest cached steps (t_last = -1 when
 *    empty).
 *  - model: the model of step t and partition `part`, owned by the window:
 *    valid until step t leaves it (or the next push, for the newest step,
 *    which freezes it). DVNR_E_INVALID if t is not cached.
 *  - bytes: FP16 size of the cached models (2 bytes per parameter) and the
 *    device bytes they hold.
 * All calls on one window must come from one thread at a time.             */
typedef struct dvnr_window_s* dvnr_window;
dvnr_status dvnr_window_create(const dvnr_box* boxes, int32_t n_parts, const dvnr_enc_cfg* encs,
                               const dvnr_mlp_cfg* mlp, int32_t capacity, uint64_t seed,
                               dvnr_window* out);
void dvnr_window_destroy(dvnr_window w);
dvnr_status dvnr_window_push(dvnr_window w, const float* const* vol_dev, const dvnr_train_cfg* cfg,
                             void* stream, float* final_loss_host, int64_t* t_out);
dvnr_status dvnr_window_range(dvnr_window w, int64_t* t_first, int64_t* t_last);
dvnr_status dvnr_window_model(dvnr_window w, int64_t t, int32_t part, dvnr_model* out);
dvnr_status dvnr_window_bytes(dvnr_window w, int64_t* model_bytes, int64_t* device_bytes);

/* Direct volume rendering from the networks (Sec. 4.3: the renderer infers
 * the models at the ray samples instead of decoding them to grids, keeping
 * the memory footprint of the compressed form). Camera, samples, transfer
 * function and compositing as dvnr_render; the value of a sample is its
 * block's network evaluated at the sample position (mapped into the block's
 * unit domain and clamped to it, as dvnr_decode_points), de-normalised. The
 * boxes must not overlap. All models must use one precision (the training
 * precision, or dvnr_set_precision); models may differ in encoding and MLP
 * configuration. The samples are streamed block by block through the
 * block's decoder in chunks of at most 2^24. Work memory: 16 bytes per
 * (pixel, block) pair whose ray crosses the block plus 4 bytes per sample
 * of a chunk (FP32 models: 16), allocated stream-ordered and released
 * before return. Synchronises the stream. Errors: DVNR_E_INVALID
 * (arguments, mixed precisions or configurations), DVNR_E_UNSUPPORTED,
 * DVNR_E_CUDA.                                                               */
dvnr_status dvnr_render_inr(const dvnr_model* models, int32_t n, const dvnr_tf* tf,
                            int32_t w, int32_t h, int32_t spr, float* rgba_dev,
                            void* stream);

/* FP64 reduction of the reconstruction error between two float32 arrays
 * (Sec. 5: PSNR from the mean squared error): out_host[0] = sum of squared
 * differences, out_host[1] = max absolute difference. Synchronises.       */
dvnr_status dvnr_error_stats(const float* a_dev, const float* b_dev, int64_t n,
                             double* out_host, void* stream);

/* Allocation-free variant of dvnr_error_stats (the paper has no counterpart;
 * this call exists for library users). For callers that must not allocate
 * device memory when they ask for the error: an in situ pipeline whose
 * simulation has reserved the device memory for itself, or a time step that
 * must not pay the implicit device synchronisation of cudaMalloc/cudaFree.
 * Same results as dvnr_error_stats (up to the order of the FP64 additions):
 * out_host[0] = sum of squared differences, out_host[1] = max |a - b|.
 *  - Scratch: a fixed device array inside the library (64 KiB + 16 B per
 *    GPU that loads the library, held until the process exits); the call
 *    allocates nothing.
 *  - Limit: n <= 2^28 (268435456) elements; larger n returns DVNR_E_INVALID
 *    with a message, before any device work.
 *  - The scratch address is looked up once per device, by dvnr_create on its
 *    device or else by the first call on a device (the device must be
 *    current).
 *  - All calls share the scratch array and leave their partial sums in it;
 *    calls whose kernels overlap on the GPU (e.g. on two streams) race and
 *    must be serialised by the caller.
 *  - Synchronises `stream`.                                                 */
dvnr_status dvnr_error_stats_noalloc(const float* a_dev, const float* b_dev, int64_t n,
                                     double* out_host, void* stream);

/* Table indices of the 8 cell corners per level for n fixed-point
 * coordinates (the indices the training and decoding kernels gather):
 * idx_dev is n x n_levels x 8, corner k = (k&1, (k>>1)&1, (k>>2)&1).       */
dvnr_status dvnr_corner_indices(dvnr_model m, const uint32_t* coords_dev,
                                int64_t n, uint32_t* idx_dev, void* stream);

/* Kernel timing for measurement: while enabled, every library kernel launch
 * is bracketed by CUDA events recorded on the stream it is launched on, and
 * the FP16 path launches its steps directly instead of replaying a CUDA
 * graph. Off by default; enabling clears the accumulators.                */
dvnr_status dvnr_profile_enable(int32_t on);

/* Total device time (ms, sum over launches) and launch count of the kernels
 * called `kernel` since profiling was enabled ("*" = every kernel).
 * Synchronises the device. Unknown names report 0 launches.               */
dvnr_status dvnr_profile_read(const char* kernel, double* total_ms, int64_t* launches);

/* Number of kernels this library has launched since it was loaded; a CUDA
 * graph replay adds the kernel nodes it runs. The body runs of the
 * early-stop training loop (a conditional graph node) are counted on the
 * device: they are included once the stream that ran them has been
 * synchronised.                                                            */
int64_t dvnr_launch_count(void);

/* How the FP16 grouped training has run its steps since the library was
 * loaded: CUDA graphs captured (each also instantiated), graph launches, and
 * steps launched directly (each pointer may be NULL). A call of n steps
 * replays graphs of 32 steps, then of 16, 8 and 4 for the binary digits of
 * the rest, each captured on its first use for the call's models and
 * settings; fewer than 4 remaining steps run directly, as does every step while
 * profiling or a lowered wait limit is active. The early-stop loop graph
 * counts one launch per call. Host counters, no synchronisation.           */
dvnr_status dvnr_graph_stats(int64_t* captures, int64_t* replays, int64_t* eager_steps);

/* Launches of the two FP16 training kernels enqueued by the host since the
 * library was loaded (each pointer may be NULL): `plain`, the kernel whose
 * 128 threads per CTA alternate gathers, tensor-core products and
 * reductions (two CTAs per SM); `ws`, the warp-specialised kernel whose CTA
 * (one per SM) runs the tensor-core chain on four warps while two groups of
 * four gather and reduce alternate tiles. A launch
 * made during graph capture counts once, its replays not at all. Calls use
 * the plain kernel unless the environment variable DVNR_TRAIN_WS=1 selects
 * the warp-specialised one wherever its layout fits (two features per
 * level, an encoding of at most 64 values, 227 KB of shared memory and 512
 * TMEM columns), including the single-step calls dvnr_train_grad and
 * dvnr_backward. Host counters, no synchronisation.                      */
dvnr_status dvnr_train_kernel_stats(int64_t* plain, int64_t* ws);

/* Diagnostic for tests of the failure path: the limit, in SM clocks, of the
 * first tensor-core wait of every CTA of the FP16 training and decoding
 * kernels (later waits keep theirs, about 2 s). cycles >= 0 sets it; 0 gives
 * up unless the first product is complete when the CTA first looks, which
 * makes that wait run out. -1 restores the default. On giving up a CTA lets
 * its product finish (bounded wait), frees its tensor memory and returns; the
 * model's step is skipped by Adam (parameters and moments unchanged, loss
 * scale kept) and the call reports DVNR_E_TIMEOUT (dvnr_train with
 * final_loss_host, dvnr_get_state). While a limit is set, FP16 training
 * launches its steps directly (no CUDA graph, no launch-shape trials).
 * Process-wide; *previous (may be NULL) receives the limit it replaces.
 * DVNR_E_INVALID for cycles < -1.                                            */
dvnr_status dvnr_debug_first_wait(int64_t cycles, int64_t* previous);

/* Measurement of the memory-request pattern of one FP16 training step of
 * model m (the training kernel is bound by scattered L1/L2 requests, not by
 * DRAM bandwidth or the tensor cores): the same Philox samples (seed 7,
 * iteration k for the k-th launch), trilinear volume reads of vol_dev (m's
 * stored block), staged gathers of the FP16 table corners and vector
 * reductions into a scratch FP32 gradient as the training kernel issues
 * them for `batch` samples, tile by tile over a persistent grid of 128-thread
 * CTAs, with no MLP. mode: bit 0 gathers, bit 1 reductions, bit 2 volume
 * reads. At most ctas_per_sm CTAs run per SM (1..16; fewer when registers or
 * shared memory do not allow them). One untimed launch, then `iters` timed
 * with CUDA events: ms_out[0] = mean ms per launch, ms_out[1] = CTAs per SM
 * that ran. The model is not changed. Needs 2 features per level and at
 * most 64 encoding values (else DVNR_E_UNSUPPORTED). Synchronises the
 * device's default stream.                                                  */
dvnr_status dvnr_probe_requests(dvnr_model m, const float* vol_dev, int32_t batch, int32_t ctas_per_sm,
                                int32_t mode, int32_t iters, double* ms_out);

/* Diagnostics for tests of the cleanup paths. Every device allocation the
 * library makes (models, workspaces, graph caches, per-call temporaries)
 * goes through one counted layer.
 *  - fail_alloc: the nth device allocation from now fails as if the device
 *    were out of memory (the call reports DVNR_E_OOM and releases what it
 *    had allocated); nth = 0 disarms. Process-wide; the countdown is
 *    consumed by the allocation it reaches. DVNR_E_INVALID for nth < 0.
 *  - live_allocs: the number and bytes of device allocations the library
 *    holds now (count and bytes may be NULL).                               */
dvnr_status dvnr_debug_fail_alloc(int64_t nth);
dvnr_status dvnr_debug_live_allocs(int64_t* count, int64_t* bytes);

/* Diagnostic of the tensor-core operand layouts used by the FP16 path: one
 * 128 x 64 x 64 tcgen05 product per operand order (A K-major/MN-major x
 * B K-major/MN-major) on values exact in FP16 and FP32, compared with a SIMT
 * product. mismatches_host[0..3] receive the number of differing outputs of
 * each case, mismatches_host[4] is 1 if a bounded wait gave up. Synchronises.
 * Returns DVNR_E_TIMEOUT if a wait gave up.                                */
dvnr_status dvnr_selftest_umma(int32_t* mismatches_host);

#ifdef __cplusplus
}
#endif
#endif /* DVNR_H */
