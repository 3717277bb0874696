/*
 * dvnr_oracle.h -- plain, slow, FP64 CPU oracle of the DVNR hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code. The product library
 * never links, includes or calls it, and it shares no code with the CUDA
 * path (it has its own Philox, hash, sampler, MLP, Adam, decode and render).
 *
 * Every function states the passage of the paper (arXiv 2304.10516, "DVNR")
 * or of the cited hash-encoding paper (Mueller et al. 2022, "Instant neural
 * graphics primitives") that it follows. Where the paper is silent the
 * reading used is stated next to the code.
 *
 * Parity pins: see tests/test_oracle_*.py. No function here is unpinned.
 */
#ifndef DVNR_ORACLE_H
#define DVNR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LEVELS 32
#define ORC_MAX_HIDDEN 8
#define ORC_QTAB 4096 /* segments of the half-normal quantile table */

/* Encoding + MLP configuration and the derived parameter layout.
 * Parameter vector theta (one model):
 *   tables  : level 0 .. L-1, each T_l entries x F features, F contiguous
 *   weights : W_0 [width x in_dim], W_1..W_{H-1} [width x width],
 *             w_out [1 x width]; every matrix row-major [out][in].           */
typedef struct {
  int32_t L, F, log2T, base_res;
  double growth;
  int32_t width, n_hidden;
  /* derived by orc_cfg_init */
  int32_t in_dim;
  int32_t N[ORC_MAX_LEVELS];      /* grid resolution of level l            */
  int32_t dense[ORC_MAX_LEVELS];  /* 1: (N+1)^3 <= T, stored densely       */
  int64_t entries[ORC_MAX_LEVELS];/* T_l                                    */
  int64_t offset[ORC_MAX_LEVELS]; /* first parameter of level l            */
  int64_t w_off[ORC_MAX_HIDDEN + 1]; /* first parameter of each matrix     */
  int64_t n_enc, n_mlp, n_params;
} orc_cfg;

/* Training hyper-parameters (Sec. 3.2, 3.3, 3.6). */
typedef struct {
  double lr, beta1, beta2, eps, weight_decay;
  double lambda_bnd, sigma_bnd;
  int32_t batch;
  int32_t loss;        /* 0 = L1 (paper), 1 = L2 (for finite differences) */
  int32_t mixed;       /* 1 = emulate the FP16 rounding points of the MP path */
  int32_t growth_interval; /* loss-scale doubling interval (MP only)      */
  uint64_t seed;
  uint32_t model;      /* model slot in the grouped call (RNG key)        */
} orc_train_cfg;

/* Per-model optimiser state carried between steps. */
typedef struct {
  double loss_scale;   /* S, 1 for the FP32 path                          */
  int64_t adam_t;      /* completed (non-skipped) Adam steps              */
  int64_t iter;        /* iterations drawn (RNG counter)                  */
  int64_t good_steps;  /* consecutive finite steps since the last change  */
  int64_t skipped;     /* steps skipped for non-finite gradients          */
} orc_state;

int  orc_cfg_init(orc_cfg* c, int32_t L, int32_t F, int32_t log2T,
                  int32_t base_res, double growth, int32_t width,
                  int32_t n_hidden);

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

double orc_round_half(double x);

uint32_t orc_corner_index(const orc_cfg* c, int level, int64_t x, int64_t y,
                          int64_t z);

void orc_init_params(const orc_cfg* c, uint64_t seed, double* theta);

void orc_quantile_table(double sigma, int64_t* tab /* ORC_QTAB + 1 */);

int  orc_sample(uint64_t seed, uint32_t model, uint64_t iter, int32_t batch,
                double lambda_bnd, const int64_t* qtab, uint32_t* m_out);

double orc_volume_trilinear(const float* vol, int64_t nx, int64_t ny,
                            int64_t nz, const uint32_t m[3]);

void orc_encode(const orc_cfg* c, const double* theta, const uint32_t m[3],
                int mixed, double* x0);

void orc_encode_batch(const orc_cfg* c, const double* theta, int64_t n,
                      const uint32_t* m, int mixed, double* x0);

void orc_targets(const float* vol, int64_t nx, int64_t ny, int64_t nz,
                 int64_t n, const uint32_t* m, double vmin, double vmax,
                 double* out);

double orc_fwd_bwd(const orc_cfg* c, const double* theta, int64_t n,
                   const uint32_t* m, const double* target, int32_t loss,
                   int32_t mixed, double loss_scale, int64_t grad_norm_count,
                   const uint8_t* flip, double* grad_enc, double* grad_mlp,
                   double* y_out, double* dx0_out, double* margin_out,
                   double* zabs_out);

void orc_adam(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
              double* theta, double* mom1, double* mom2, const double* grad);

double orc_train(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
                 double* theta, double* mom1, double* mom2, const float* vol,
                 int64_t nx, int64_t ny, int64_t nz, double vmin, double vmax,
                 int64_t steps, double* loss_hist);

/* Iteration budget of one training call (Sec. 3.2): the fixed count `steps`,
 * or ceil(n_vox / batch) * epochs when epochs > 0, raised to min_steps:
 * N_train^max = max(N_train^min, ceil(N_vox / N_batch) N_epoch).            */
int64_t orc_max_iterations(int64_t n_vox, int64_t batch, int64_t steps,
                           int64_t epochs, int64_t min_steps);

/* Adaptive table size and base resolution of a partition (Sec. 3.2):
 * T = max(T_min, T_ref N_vox / N_vox^global rounded up to a power of two)
 * and R_0 = floor(R_ref (T / T_ref)^(1/3)), at least 1. T_ref = 2^log2_T_ref,
 * T_min = 2^log2_T_min. Writes log2 T and R_0.                              */
void orc_adaptive_encoding(int64_t n_vox, int64_t n_vox_global, int32_t log2_T_ref,
                           int32_t log2_T_min, double R_ref, int32_t* log2_T,
                           int32_t* base_res);

/* Early stop (Sec. 3.2) over a recorded loss sequence: the moving average
 * m_1 = L_1, m_t = d m_{t-1} + (1 - d) L_t over the finite steps (finite[t]
 * != 0; a step whose gradient was non-finite leaves m unchanged), stopping
 * after the first step with m_t < stop_loss (stop_loss 0: never). Returns
 * the number of steps run (n if it never stops); *ema_out = m after them
 * (-1 if no finite step).                                                   */
int64_t orc_stop_step(const double* losses, const int32_t* finite, int64_t n,
                      double decay, double stop_loss, double* ema_out);

/* orc_train under the budget and early stop of one call: at most `budget`
 * iterations, ending after the first whose moving average falls below
 * stop_loss. Returns the iterations run; loss_hist (budget entries, may be
 * NULL) receives their losses, *ema_out the final moving average and
 * *stopped_out 1 if the threshold ended the call.                            */
int64_t orc_train_budget(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
                         double* theta, double* mom1, double* mom2, const float* vol,
                         int64_t nx, int64_t ny, int64_t nz, double vmin, double vmax,
                         int64_t budget, double stop_loss, double decay,
                         double* loss_hist, double* ema_out, int32_t* stopped_out);

void orc_decode_unit(const orc_cfg* c, const double* theta, int64_t n,
                     const uint32_t* m, int mixed, double vmin, double vmax,
                     double* out);

uint32_t orc_grid_coord(int64_t j, int64_t n);

void orc_decode_grid(const orc_cfg* c, const double* theta, const int64_t n[3],
                     int32_t ghost, int mixed, double vmin, double vmax,
                     double* out);

void orc_render(int32_t n_blocks, const double* const* grids,
                const int64_t* lo, const int64_t* hi, const double* tf,
                int32_t w, int32_t h, int32_t spr, double* rgba);

/* Direct volume rendering from the networks (Sec. 4.3): the camera, samples,
 * transfer function and compositing of orc_render, with the value of a
 * sample taken from its block's network at the sample position (global
 * voxel coordinates mapped to the block's unit domain, clamped, rounded to
 * the 2^-24 lattice) and de-normalised with the block's value range. Only
 * the n_pix pixels listed in pix (index py * w + px) are rendered, into
 * rgba[4 i ...]. thetas/vmin/vmax/ghost per block; one configuration.    */
void orc_render_inr(const orc_cfg* c, int32_t n_blocks, const double* const* thetas,
                    const int64_t* lo, const int64_t* hi, const int32_t* ghost,
                    int mixed, const double* vmin, const double* vmax,
                    const double* tf, int32_t w, int32_t h, int32_t spr,
                    int64_t n_pix, const int64_t* pix, double* rgba);

double orc_mse(const double* a, const float* b, int64_t n, double* max_abs);

int  orc_threads(void);
int  orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
