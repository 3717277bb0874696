// mp_path.cu -- the FP16 tensor-core path of libdvnr.
//
// Training (Sec. 3.2): one persistent kernel per step trains every model of
// the call (the paper's one-model-per-partition, Sec. 3.1, as a grouped
// launch): each CTA walks a contiguous run of 128-sample tiles, and per tile
//   draw samples (Philox) -> trilinear target -> hash-grid gather (FP16
//   tables, FP32 interpolation) -> MLP forward on tcgen05 (FP16 operands in
//   shared memory, FP32 accumulators in TMEM) -> L1/L2 loss with loss scale
//   -> backward on tcgen05: dL/dH per layer, and the weight gradients of the
//   whole run accumulated in TMEM -> dL/d(encoding) scattered into the FP32
//   table gradients with vector atomics. When the run leaves a model, the
//   CTA adds its accumulated weight gradients and loss to the model's.
// The tiles of a step go in L2-sized waves; the fused Adam of util.cu
// follows, and 32 steps are replayed from one CUDA graph. A call whose models
// can leave the group (per-model budgets, the moving-average stop) runs as
// one graph launch whose conditional WHILE node repeats the 32 steps until
// no model is active. Decoding (Sec. 3, Sec. 4.1) runs the forward half on
// the same tiles, at grid points, given points or the samples of a ray
// lattice (direct rendering, Sec. 4.3), with one ACT tile that each layer's
// outputs overwrite.
//
// Tile buffers in shared memory hold 128 samples x features as FP16 core
// matrices (8 samples x 8 features, 128 B): feature group g, sample group q
// at byte ((g * 16) + q) * 128. Read along features they are the K-major A
// operand of a layer (M = samples); read along samples they are the MN-major
// operands of the weight-gradient products (K = samples).
//   ACT: X0 (the encoding, D features), H_1 .. H_{H-1} (W features each)
//   DZ : dZ_1 .. dZ_H (W features each)
// dW_k = dZ_{k+1}^T H_k is formed as an M = 128 product whose A operand is
// the 128 features starting at dZ_{k+1}; rows W..127 of that accumulator
// collect unused products and are never read.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mp_common.cuh"
#include "mp_path.cuh"

namespace dvnr {

namespace {

#ifndef DVNR_TRAIN_STAGED
#define DVNR_TRAIN_STAGED 1
#endif
// Step graphs of the grouped training: 2^kMaxGraphLog steps per replay (and
// per body run of the early-stop loop); the fixed graphs of a call's
// remaining steps have 2^k steps, k >= kMinGraphLog (fewer steps run
// eagerly: a graph of one or two steps saves less than its capture costs a
// one-off call). A call of n steps thus replays graphs for the binary digits
// of n down to 4, captured the first time they are needed.
constexpr int kMaxGraphLog = 5;
constexpr int kMinGraphLog = 2;

// Limit of each CTA's first tensor-core wait in the training and decoding
// kernels (dvnr_debug_first_wait); kWaitCycles unless a test lowers it.
std::atomic<long long> g_first_wait{kWaitCycles};

// Revision of the training kernel's memory behaviour; the DRAM-traffic figure
// of an Nsight Compute capture is reported only while it matches.
[[maybe_unused]] constexpr int kTrainKernelRevision = 12;

struct MpModel {
  const __half* theta16;
  float* grad;
  const float* vol;
  int32_t nx, ny, nz;
  uint32_t slot;
  ModelState* st;
};

struct MpParams {
  LevelTab lv;
  int32_t D, H;
  int64_t w_off[kMaxHidden + 1];
  MpLayout lay;
  int32_t batch, n_bnd, loss, tiles_per_model;
  int64_t total_tiles;
  uint2 key;
  const int32_t* qtab;
  const MpModel* models;
  float inv_batch;
  int32_t explicit_iter;
  uint32_t iter;
  float loss_scale_override;
  float* dbg_y;
  float* dbg_dx0;
  float* dbg_tgt;
  uint32_t* dbg_coords;
  // the tiles of a step are taken in waves of wave_tiles: every CTA walks
  // its share of wave 0, then of wave 1, ..., so that the tables and
  // gradients in use at any time stay within L2; a wave may split a model
  int64_t wave_tiles;
  // the launch trains waves [wave_first, wave_end) of the step (wave_end < 0:
  // to the last); a step run wave by wave interleaves the Adam updates of
  // the models each wave begins (see mp_train)
  int32_t wave_first, wave_end;
  // models of the step: sched[0] = n_active, sched[1 + a] = index of the
  // a-th active model, sched[1 + n_models + m] = position of model m (-1 when
  // inactive), written by k_mp_schedule; nullptr = all n_models take part
  const int32_t* sched;
  int32_t n_models;
  // limit of each CTA's first tensor-core wait (SM clocks; <= 0: give up
  // unless complete at once); later waits use kWaitCycles
  long long first_wait_cycles;
  // backward at caller-given points (dvnr_backward; single model, no volume):
  // fixed-point coordinates (batch x 3) instead of drawn samples, the
  // upstream dL/dy (batch) instead of the loss, and the loss scale read from
  // *ext_scale; all nullptr in training
  const uint32_t* ext_coords;
  const float* ext_dy;
  const float* ext_scale;
};

struct MpDecodeParams {
  LevelTab lv;
  int32_t D, H;
  int64_t w_off[kMaxHidden + 1];
  MpLayout lay;
  const __half* theta16;
  const ModelState* st;
  int64_t n, n_tiles;
  const float* xyz;
  const uint32_t* coords;  // grid_mode 3: fixed-point coordinates, n x 3
  // 0: xyz points, 1: the owned grid, 2: ray lattice (depth-major), 3: given
  // fixed-point coordinates, the network output written without
  // de-normalisation (dvnr_forward)
  int grid_mode;
  int64_t e[3], nstore[3];
  RayFrame rf;     // grid_mode 2: the samples of rays r0 .. r0+nr-1 of block rb,
  RayBlock rb;     // point i = sample k0 + i / nr of ray r0 + i % nr
  int64_t r0, nr;
  int32_t ghost;
  float origin[3];
  float* out;
  // the launch's divisors: e[0], e[1] (grid point -> voxel), 2 (nstore[a] - 1)
  // (voxel -> fixed point), nr and rb.npx (ray lattice)
  FastDiv div_e0, div_e1, div_fix[3], div_nr, div_npx;
  long long first_wait_cycles;  // as MpParams
};

template <int F>
__device__ __forceinline__ bool scatter_from_tmem(const LevelTab& lv, float* __restrict__ grad,
                                                  uint3 m, bool valid, uint32_t tl,
                                                  float* dbg_row, float inv_S) {
  bool bad = false;
  const int D = lv.in_dim;
  int c = 0;
  for (; c < D; c += 16) {
    float d[16];
    umma::ld16(tl + (uint32_t)c, d);
    umma::ld_wait();
    if (!valid) continue;
    if (dbg_row) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c + j < D) dbg_row[c + j] = d[j] * inv_S;
    }
    // whole chunks of real levels, then a last chunk that ends in padding
    if (c + 16 <= D)
      bad |= scatter_chunk<F, false>(lv, grad, m, d, c);
    else
      bad |= scatter_chunk<F, true>(lv, grad, m, d, c);
  }
  return bad;
}

// ------------------------------------------------------- training kernel ---
template <int W, int F>
__global__ void __launch_bounds__(kTile, 1) k_mp_train(const __grid_constant__ MpParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 8);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(smem + 12);
  uint8_t* s_act = smem + p.lay.smem_act;
  uint8_t* s_dz = smem + p.lay.smem_dz;
  const float* s_wout = reinterpret_cast<const float*>(smem + p.lay.smem_wout);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = p.D, H = p.H;
  // the step's active models (uniform over the grid; nothing to do when every
  // model has spent its budget or stopped)
  const int n_act = p.sched ? p.sched[0] : p.n_models;
  if (n_act <= 0) return;
  const int64_t T_act = (int64_t)n_act * p.tiles_per_model;
  const int n_waves = (int)((T_act + p.wave_tiles - 1) / p.wave_tiles);

  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    *abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, p.lay.tmem_cols);
  // the zero padding of X0 (features D .. dpad-1): nothing else writes it
  if ((int)p.lay.dpad > D) zero_pad_rows<F>(D, (int)p.lay.dpad, s_act, (uint32_t)tid);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's TMEM lanes
  uint32_t phase = 0;

  int cur = -1;
  bool first_tile = true;
  MpModel md{};
  SampleParams sp;
  sp.key = p.key;
  sp.n_bnd = p.n_bnd;
  sp.qtab = p.qtab;
  uint32_t iter = 0;
  float S = 1.f, vmin = 0.f, inv_range = 0.f;
  constexpr int NOUT = W >= 32 ? W / 32 : 1;
  float acc_out[NOUT];
  float loss_acc = 0.f;
  // the next tile's sample and volume corners, drawn and fetched while the
  // tensor core runs this tile's first product (when the next tile is of
  // the same model and in this CTA's run of the wave)
  bool have_next = false;
  uint3 mc_next = make_uint3(0u, 0u, 0u);
  VolCorners vc_next{};

  // thread 0: an MMA was committed and its completion not yet seen by
  // thread 0 (after an abort, teardown waits for it before freeing TMEM)
  bool inflight = false;
  long long wait_limit = p.first_wait_cycles;
  // wait for the tensor core and raise/observe the CTA-wide abort flag
  auto mma_wait = [&]() -> bool {
    if (umma::mbar_wait_bounded(mbar, phase, abort_flag, wait_limit)) inflight = false;
    wait_limit = kWaitCycles;
    phase ^= 1u;
    __syncthreads();
    return *abort_flag == 0u;
  };

  // add the run's weight gradients and loss of the current model to the
  // model's MLP gradient and loss sum (16-byte vector reductions; every CTA
  // whose run touched the model adds its share, Adam clears them)
  auto flush = [&]() {
    umma::fence_after_sync();
    float* part = md.grad + p.w_off[0];
    if (warp * 32 < W) {
      const int r = warp * 32 + lane;  // output row of the layer
      for (int k = 0; k < H; ++k) {
        const int in = k == 0 ? D : W;
        float* g = part + (p.w_off[k] - p.w_off[0]);
        for (int c = 0; c < in; c += 16) {
          float v[16];
          umma::ld16(tl + p.lay.dw_col[k] + c, v);
          umma::ld_wait();
          if (r < W && (in & 15) == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) red_add<4>(g + (size_t)r * in + c + 4 * j, v + 4 * j);
          } else if (r < W) {
            // columns past D (layer 0's zero padding) are dropped; a row of
            // D % 4 != 0 inputs is not 16-byte aligned: scalar adds
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int c0 = c + 4 * j;
              if (c0 + 4 <= in && (in & 3) == 0) {
                red_add<4>(g + (size_t)r * in + c0, v + 4 * j);
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (c0 + e < in) atomicAdd(g + (size_t)r * in + c0 + e, v[4 * j + e]);
              }
            }
          }
        }
      }
    }
    // dW_out and the loss: sum the four warps through shared memory (the
    // DZ tile is idle here)
    float* s_red = reinterpret_cast<float*>(s_dz);
    if (W >= 32) {
#pragma unroll
      for (int j = 0; j < NOUT; ++j) s_red[warp * (W + 1) + NOUT * lane + j] = acc_out[j];
    } else if (!(lane & 1)) {
      s_red[warp * (W + 1) + (lane >> 1)] = acc_out[0];
    }
    float l = loss_acc;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) s_red[warp * (W + 1) + W] = l;
    __syncthreads();
    if (tid <= W) {
      const float t = s_red[tid] + s_red[(W + 1) + tid] + s_red[2 * (W + 1) + tid] + s_red[3 * (W + 1) + tid];
      if (tid < W)
        atomicAdd(part + (p.w_off[H] - p.w_off[0]) + tid, t);
      else
        atomicAdd(&md.st->loss_sum, t);
    }
    umma::fence_before_sync();
    __syncthreads();
  };

  // tiles are numbered over the active models in order (position a covers
  // tiles [a tpm, (a + 1) tpm)); the waves split that sequence
  const int wv_end = p.wave_end < 0 ? n_waves : min(p.wave_end, n_waves);
  for (int wv = p.wave_first; wv < wv_end; ++wv) {
  const int64_t wb = (int64_t)wv * p.wave_tiles;
  const int64_t Tw = p.wave_tiles < T_act - wb ? p.wave_tiles : T_act - wb;
  const int64_t g_begin = wb + (Tw * blockIdx.x) / gridDim.x;
  const int64_t g_end = wb + (Tw * (blockIdx.x + 1)) / gridDim.x;
  for (int64_t g = g_begin; g < g_end; ++g) {
    const int pos = (int)(g / p.tiles_per_model);
    const int tile = (int)(g - (int64_t)pos * p.tiles_per_model);
    const int model = p.sched ? p.sched[1 + pos] : pos;
    if (model != cur) {
      if (cur >= 0) flush();
      cur = model;
      md = p.models[model];
      sp.model = md.slot;
      iter = p.explicit_iter ? p.iter : md.st->iter;
      S = p.ext_scale ? *p.ext_scale : (p.loss_scale_override > 0.f ? p.loss_scale_override : md.st->loss_scale);
      value_range(md.st, vmin, inv_range);
#pragma unroll
      for (int j = 0; j < NOUT; ++j) acc_out[j] = 0.f;
      loss_acc = 0.f;
      first_tile = true;
      load_weights(md.theta16, p.w_off, D, H, W, p.lay, smem);
    }
    // -- sample, target, encode
    const int i = tile * kTile + tid;
    const bool valid = i < p.batch;
    uint3 mc = make_uint3(0u, 0u, 0u);
    VolCorners vc{};
    if (have_next) {
      mc = mc_next;
      vc = vc_next;
    } else {
      if (valid)
        mc = p.ext_coords ? make_uint3(p.ext_coords[3 * i], p.ext_coords[3 * i + 1], p.ext_coords[3 * i + 2])
                          : draw_sample(sp, (uint32_t)i, iter);
      if (valid && md.vol) vc = vol_fetch(md.vol, md.nx, md.ny, md.nz, mc);  // in flight during the encode
    }
    have_next = false;
#if DVNR_TRAIN_STAGED
    if constexpr (F == 2) {
      // all gathers of the tile in flight at once, staged in the dZ tile and
      // the hidden-activation tiles (idle until the forward pass)
      encode_to_tile_staged(p.lv, md.theta16, mc, valid, s_act, (uint32_t)tid, s_dz, H * W / 16,
                            s_act + p.lay.dpad * 256u, (H - 1) * W / 16);
    } else
#endif
      encode_to_tile<F, DVNR_TRAIN_PAIR>(p.lv, md.theta16, mc, valid, s_act, (uint32_t)tid);
    const float target = (valid && md.vol) ? (vol_interp(vc) - vmin) * inv_range : 0.f;
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();

    // -- forward: H_{k+1} = ReLU(H_k W_k^T)
    float h[W];
    uint64_t maskH = 0;
    for (int k = 0; k < H; ++k) {
      if (tid == 0) {
        umma::fence_after_sync();
        issue_forward(tmem, smem, p.lay, k, k == 0 ? (int)p.lay.dpad : W, W);
        umma::commit(mbar);
        inflight = true;
      }
      if (k == 0 && g + 1 < g_end) {
        const int pos_n = (int)((g + 1) / p.tiles_per_model);
        const int model_n = p.sched ? p.sched[1 + pos_n] : pos_n;
        if (model_n == cur) {
          const int i_n = (int)(g + 1 - (int64_t)pos_n * p.tiles_per_model) * kTile + tid;
          const bool valid_n = i_n < p.batch;
          mc_next = make_uint3(0u, 0u, 0u);
          if (valid_n)
            mc_next = p.ext_coords ? make_uint3(p.ext_coords[3 * i_n], p.ext_coords[3 * i_n + 1],
                                                p.ext_coords[3 * i_n + 2])
                                   : draw_sample(sp, (uint32_t)i_n, iter);
          vc_next = VolCorners{};
          if (valid_n && md.vol) vc_next = vol_fetch(md.vol, md.nx, md.ny, md.nz, mc_next);
          have_next = true;
        }
      }
      if (!mma_wait()) goto teardown;
      umma::fence_after_sync();
#pragma unroll
      for (int c = 0; c < W / 16; ++c) {
        float v[16];
        umma::ld16(tl + c * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) h[c * 16 + j] = v[j];
      }
      umma::ld_wait();
      if (k < H - 1) {
        const uint32_t f0 = p.lay.act_off[k + 1];
#pragma unroll
        for (int c = 0; c < W / 8; ++c) {
          uint4 u;
          uint32_t* pu = &u.x;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            __half2 t = __floats2half2_rn(fmaxf(h[c * 8 + 2 * j], 0.f), fmaxf(h[c * 8 + 2 * j + 1], 0.f));
            pu[j] = *reinterpret_cast<uint32_t*>(&t);
          }
          *reinterpret_cast<uint4*>(s_act + tile_off(f0 + c * 8, tid)) = u;
        }
        umma::fence_proxy_async();
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (h[j] > 0.f) maskH |= 1ull << j;
          h[j] = __half2float(__float2half_rn(fmaxf(h[j], 0.f)));
        }
      }
      umma::fence_before_sync();
      __syncthreads();
    }

    {
      // -- output, loss, dL/dy (scaled by S)
      float y = 0.f;
#pragma unroll
      for (int j = 0; j < W; ++j) y += h[j] * s_wout[j];
      float dy = 0.f;
      if (valid && p.ext_dy) {
        dy = p.ext_dy[i] * S;
        if (!isfinite(y)) atomicOr(&md.st->overflow, 1u);
      } else if (valid) {
        const float d = y - target;
        if (p.loss == DVNR_LOSS_L1) {
          loss_acc += fabsf(d);
          dy = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * (S * p.inv_batch);
        } else {
          loss_acc += d * d;
          dy = 2.f * d * (S * p.inv_batch);
        }
        if (!isfinite(y)) atomicOr(&md.st->overflow, 1u);
        if (p.dbg_y && cur == 0) {
          p.dbg_y[i] = y;
          p.dbg_tgt[i] = target;
          p.dbg_coords[3 * i] = mc.x;
          p.dbg_coords[3 * i + 1] = mc.y;
          p.dbg_coords[3 * i + 2] = mc.z;
        }
      }
      // dW_out += fp16(dy) h_H, reduced over the warp (reduce-scatter)
      {
        const float dy16 = __half2float(__float2half_rn(dy));
        float v[W];
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = dy16 * h[j];
        int n = W;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
          if (n > 1) {
            const bool upper = (lane & s) != 0;
            const int half = n / 2;
#pragma unroll
            for (int j = 0; j < W / 2; ++j) {
              if (j < half) {
                const float send = upper ? v[j] : v[j + half];
                const float keep = upper ? v[j + half] : v[j];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
              }
            }
            n = half;
          } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], s);
          }
        }
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc_out[j] += v[j];
      }
      // dZ_H = fp16(dy w_out) where z_H > 0
      const uint32_t f0 = (uint32_t)(H - 1) * W;
#pragma unroll
      for (int c = 0; c < W / 8; ++c) {
        uint4 u;
        uint32_t* pu = &u.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int a = c * 8 + 2 * j;
          const float v0 = ((maskH >> a) & 1ull) ? dy * s_wout[a] : 0.f;
          const float v1 = ((maskH >> (a + 1)) & 1ull) ? dy * s_wout[a + 1] : 0.f;
          __half2 t = __floats2half2_rn(v0, v1);
          pu[j] = *reinterpret_cast<uint32_t*>(&t);
        }
        *reinterpret_cast<uint4*>(s_dz + tile_off(f0 + c * 8, tid)) = u;
      }
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();

    // -- backward: layer k maps H_{k-1} -> Z_k with W_{k-1}
    {
      for (int k = H; k >= 1; --k) {
        const int in = k == 1 ? (int)p.lay.dpad : W;  // layer 0's K includes the zero padding
        if (tid == 0) {
          umma::fence_after_sync();
          const uint32_t dz0 = umma::smem_u32(s_dz) + ((uint32_t)((k - 1) * W) >> 3) * 2048u;
          const uint32_t act0 = umma::smem_u32(s_act) + (p.lay.act_off[k - 1] >> 3) * 2048u;
          // dW_{k-1} += dZ_k^T H_{k-1} (K = samples; both operands MN-major)
          const uint32_t idw = umma::idesc_f16(kTile, in, 1, 1);
          for (int ks = 0; ks < kTile / 16; ++ks) {
            const uint64_t a = umma::sdesc(dz0 + ks * 256u, 128u, 2048u);
            const uint64_t b = umma::sdesc(act0 + ks * 256u, 128u, 2048u);
            umma::mma_f16(tmem + p.lay.dw_col[k - 1], a, b, idw, (first_tile && ks == 0) ? 0u : 1u);
          }
          // dH_{k-1} = dZ_k W_{k-1} (A K-major over the W outputs, B MN-major)
          const uint32_t ibw = umma::idesc_f16(kTile, in, 0, 1);
          const uint32_t w0 = umma::smem_u32(smem + p.lay.smem_w + p.lay.wbyte[k - 1]);
          const uint32_t wb = (uint32_t)(W >> 3) * 128u;
          for (int kk = 0; kk < W / 16; ++kk) {
            const uint64_t a = umma::sdesc(dz0 + kk * 4096u, 2048u, 128u);
            const uint64_t b = umma::sdesc(w0 + kk * 256u, 128u, wb);
            umma::mma_f16(tmem, a, b, ibw, kk > 0);
          }
          umma::commit(mbar);
          inflight = true;
        }
        if (!mma_wait()) goto teardown;
        umma::fence_after_sync();
        if (k > 1) {
          float dh[W];
#pragma unroll
          for (int c = 0; c < W / 16; ++c) {
            float v[16];
            umma::ld16(tl + c * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) dh[c * 16 + j] = v[j];
          }
          umma::ld_wait();
          const uint32_t fa = p.lay.act_off[k - 1], fz = (uint32_t)(k - 2) * W;
#pragma unroll
          for (int c = 0; c < W / 8; ++c) {
            const uint4 hv = *reinterpret_cast<const uint4*>(s_act + tile_off(fa + c * 8, tid));
            const uint32_t* ph = &hv.x;
            uint4 u;
            uint32_t* pu = &u.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const __half2 hh = *reinterpret_cast<const __half2*>(ph + j);
              const float2 hf = __half22float2(hh);
              const float v0 = hf.x > 0.f ? dh[c * 8 + 2 * j] : 0.f;
              const float v1 = hf.y > 0.f ? dh[c * 8 + 2 * j + 1] : 0.f;
              __half2 t = __floats2half2_rn(v0, v1);
              pu[j] = *reinterpret_cast<uint32_t*>(&t);
            }
            *reinterpret_cast<uint4*>(s_dz + tile_off(fz + c * 8, tid)) = u;
          }
          umma::fence_proxy_async();
          umma::fence_before_sync();
          __syncthreads();
        }
      }
      // -- scatter dL/d(encoding) (still in TMEM columns 0..D-1) into the table gradients
      float* dbg_row = (p.dbg_dx0 && cur == 0 && valid) ? p.dbg_dx0 + (size_t)i * D : nullptr;
      if (scatter_from_tmem<F>(p.lv, md.grad, mc, valid, tl, dbg_row, 1.0f / S))
        atomicOr(&md.st->overflow, 1u);
      umma::fence_before_sync();
    }
    first_tile = false;
  }
  }
  if (cur >= 0) flush();

teardown:
  if (*abort_flag) {
    if (tid == 0) {
      // give the MMA whose wait gave up a bounded chance to finish before
      // TMEM is freed: its phase is the one before `phase` (flipped on exit
      // from the wait)
      if (inflight) {
        const long long t0 = clock64();
        while (!umma::mbar_try_wait(mbar, phase ^ 1u) && clock64() - t0 < kWaitCycles) {
        }
      }
      // the step of this model is incomplete: count the timeout and have Adam
      // skip the step (kStepAborted), which also clears the partial gradient
      if (cur >= 0) {
        atomicAdd(&md.st->timeouts, 1u);
        atomicOr(&md.st->overflow, kStepAborted);
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, p.lay.tmem_cols);
}

// ------------------------------------------ warp-specialised training ---
// k_mp_train_ws: the step of k_mp_train with the memory work and the
// tensor-core chain on different warps of one CTA per SM. Warps 0-3 (the
// chain) run the tiles' forward products, loss and backward products in
// order; two gathering groups (warps 4-7 and 8-11) take alternate tiles: a
// group gathers its tile into its X0 slot, waits for the chain's products of
// that tile, then scatters the tile's dL/d(encoding) into the table
// gradients, so that one group's gathers, the other's reductions and the
// chain's products overlap. Handoffs are mbarriers: full[b] (128 arrivals: X0
// slot b, its targets and coordinates written), dx[b] (the chain's commit
// after a tile's last products: its dL/dX0 is in slot b's TMEM columns and X0
// slot b is free) and dxfree[b] (128 arrivals: slot b's dL/dX0 read back). Every wait is
// bounded; a wait that gives up raises the CTA's abort flag, and each warp
// group leaves its loop at its next group barrier, which takes the OR of its
// threads' view of the flag so that the group decides as one. Same results
// as k_mp_train up to the order of the floating-point reductions.
template <int W, int F>
__global__ void __launch_bounds__(3 * kTile, 1) k_mp_train_ws(const __grid_constant__ MpParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 8);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(smem + 12);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 16);    // [2]
  uint64_t* dxr = reinterpret_cast<uint64_t*>(smem + 32);     // [2]
  uint64_t* dxfree = reinterpret_cast<uint64_t*>(smem + 48);  // [2]
  uint64_t* fin = reinterpret_cast<uint64_t*>(smem + 64);
  volatile int32_t* mem_model = reinterpret_cast<volatile int32_t*>(smem + 72);  // [2]
  uint8_t* s_act = smem + p.lay.smem_act;
  uint8_t* s_dz = smem + p.lay.smem_dz;
  const float* s_wout = reinterpret_cast<const float*>(smem + p.lay.smem_wout);
  float* s_tgt = reinterpret_cast<float*>(smem + p.lay.smem_tgt);
  uint32_t* s_crd = reinterpret_cast<uint32_t*>(smem + p.lay.smem_crd);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool chain = tid < kTile;
  const int lt = tid & (kTile - 1);  // thread within its warp group: TMEM lane and tile sample
  const int D = p.D, H = p.H;
  const int n_act = p.sched ? p.sched[0] : p.n_models;
  if (n_act <= 0) return;
  const int64_t T_act = (int64_t)n_act * p.tiles_per_model;
  const int n_waves = (int)((T_act + p.wave_tiles - 1) / p.wave_tiles);
  const int wv_end = p.wave_end < 0 ? n_waves : min(p.wave_end, n_waves);

  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    for (int b = 0; b < 2; ++b) {
      umma::mbar_init(full + b, kTile);
      umma::mbar_init(dxr + b, 1);
      umma::mbar_init(dxfree + b, kTile);
    }
    umma::mbar_init(fin, 1);
    *abort_flag = 0u;
    mem_model[0] = mem_model[1] = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, p.lay.tmem_cols);
  // the zero padding of the X0 slots (features D .. dpad-1), each by its
  // gathering group: nothing else writes it
  if ((int)p.lay.dpad > D && !chain)
    zero_pad_rows<F>(D, (int)p.lay.dpad, smem + p.lay.smem_x0[(warp >> 2) - 1], (uint32_t)lt);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's TMEM lanes

  // the CTA's tiles in order: its share of each wave in turn; (wv, g, ge)
  // advances to the next tile, false when there is none
  auto next_tile = [&](int& wv, int64_t& g, int64_t& ge) -> bool {
    ++g;
    while (g >= ge) {
      if (++wv >= wv_end) return false;
      const int64_t wb = (int64_t)wv * p.wave_tiles;
      const int64_t Tw = p.wave_tiles < T_act - wb ? p.wave_tiles : T_act - wb;
      g = wb + (Tw * blockIdx.x) / gridDim.x;
      ge = wb + (Tw * (blockIdx.x + 1)) / gridDim.x;
    }
    return true;
  };
  auto model_of = [&](int64_t g, int& tile) -> int {
    const int pos = (int)(g / p.tiles_per_model);
    tile = (int)(g - (int64_t)pos * p.tiles_per_model);
    return p.sched ? p.sched[1 + pos] : pos;
  };
  auto scale_of = [&](const MpModel& md) -> float {
    return p.ext_scale ? *p.ext_scale : (p.loss_scale_override > 0.f ? p.loss_scale_override : md.st->loss_scale);
  };

  int cur = -1;  // the chain's model
  MpModel md{};
  if (chain) {
    // ------------------------------------------------------------ chain --
    uint32_t phase = 0;
    long long wait_limit = p.first_wait_cycles;
    auto mma_wait = [&]() -> bool {
      umma::mbar_wait_bounded(mbar, phase, abort_flag, wait_limit);
      wait_limit = kWaitCycles;
      phase ^= 1u;
      return !umma::bar_or(1, kTile, *abort_flag != 0u);
    };
    auto group_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      umma::mbar_wait_bounded(bar, parity, abort_flag, kWaitCycles);
      return !umma::bar_or(1, kTile, *abort_flag != 0u);
    };
    bool first_tile = true;
    float S = 1.f;
    constexpr int NOUT = W >= 32 ? W / 32 : 1;
    float acc_out[NOUT];
    float loss_acc = 0.f;
    // the run's weight gradients and loss of the current model into the
    // model's MLP gradient and loss sum, as k_mp_train's flush
    auto flush = [&]() {
      umma::fence_after_sync();
      float* part = md.grad + p.w_off[0];
      if (warp * 32 < W) {
        const int r = warp * 32 + lane;
        for (int k = 0; k < H; ++k) {
          const int in = k == 0 ? D : W;
          float* g = part + (p.w_off[k] - p.w_off[0]);
          for (int c = 0; c < in; c += 16) {
            float v[16];
            umma::ld16(tl + p.lay.dw_col[k] + c, v);
            umma::ld_wait();
            if (r < W && (in & 15) == 0) {
#pragma unroll
              for (int j = 0; j < 4; ++j) red_add<4>(g + (size_t)r * in + c + 4 * j, v + 4 * j);
            } else if (r < W) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int c0 = c + 4 * j;
                if (c0 + 4 <= in && (in & 3) == 0) {
                  red_add<4>(g + (size_t)r * in + c0, v + 4 * j);
                } else {
#pragma unroll
                  for (int e = 0; e < 4; ++e)
                    if (c0 + e < in) atomicAdd(g + (size_t)r * in + c0 + e, v[4 * j + e]);
                }
              }
            }
          }
        }
      }
      float* s_red = reinterpret_cast<float*>(s_dz);
      if (W >= 32) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j) s_red[warp * (W + 1) + NOUT * lane + j] = acc_out[j];
      } else if (!(lane & 1)) {
        s_red[warp * (W + 1) + (lane >> 1)] = acc_out[0];
      }
      float l = loss_acc;
      for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
      if (lane == 0) s_red[warp * (W + 1) + W] = l;
      umma::bar_sync(1, kTile);
      if (lt <= W) {
        const float t = s_red[lt] + s_red[(W + 1) + lt] + s_red[2 * (W + 1) + lt] + s_red[3 * (W + 1) + lt];
        if (lt < W)
          atomicAdd(part + (p.w_off[H] - p.w_off[0]) + lt, t);
        else
          atomicAdd(&md.st->loss_sum, t);
      }
      umma::fence_before_sync();
      umma::bar_sync(1, kTile);
    };

    int wv = p.wave_first - 1;
    int64_t g = 0, ge = 0, t = 0;
    bool go = true;
    while (go && next_tile(wv, g, ge)) {
      const int b = (int)(t & 1);
      const uint32_t use = (uint32_t)(t >> 1);
      if (!group_wait(full + b, use & 1u)) break;
      int tile;
      const int model = model_of(g, tile);
      if (model != cur) {
        if (cur >= 0) {
          // the previous tile's last products complete before the run's dW leave TMEM
          if (!group_wait(dxr + ((t - 1) & 1), (uint32_t)((t - 1) >> 1) & 1u)) break;
          flush();
        }
        cur = model;
        md = p.models[model];
        S = scale_of(md);
#pragma unroll
        for (int j = 0; j < NOUT; ++j) acc_out[j] = 0.f;
        loss_acc = 0.f;
        first_tile = true;
        load_weights(md.theta16, p.w_off, D, H, W, p.lay, smem, lt, kTile);
        umma::fence_proxy_async();
        umma::fence_before_sync();
        umma::bar_sync(1, kTile);
      }
      const int i = tile * kTile + lt;
      const bool valid = i < p.batch;
      const float target = s_tgt[b * kTile + lt];
      const uint32_t x0 = umma::smem_u32(smem + p.lay.smem_x0[b]);

      // -- forward: H_{k+1} = ReLU(H_k W_k^T)
      float h[W];
      uint64_t maskH = 0;
      for (int k = 0; k < H; ++k) {
        if (lt == 0) {
          umma::fence_after_sync();
          const uint32_t a0 = k == 0 ? x0 : umma::smem_u32(s_act) + (p.lay.act_off[k] >> 3) * 2048u;
          issue_forward_at(tmem, a0, smem, p.lay, k, k == 0 ? (int)p.lay.dpad : W, W);
          umma::commit(mbar);
        }
        if (!mma_wait()) {
          go = false;
          break;
        }
        umma::fence_after_sync();
#pragma unroll
        for (int c = 0; c < W / 16; ++c) {
          float v[16];
          umma::ld16(tl + c * 16, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) h[c * 16 + j] = v[j];
        }
        umma::ld_wait();
        if (k < H - 1) {
          const uint32_t f0 = p.lay.act_off[k + 1];
#pragma unroll
          for (int c = 0; c < W / 8; ++c) {
            uint4 u;
            uint32_t* pu = &u.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              __half2 q = __floats2half2_rn(fmaxf(h[c * 8 + 2 * j], 0.f), fmaxf(h[c * 8 + 2 * j + 1], 0.f));
              pu[j] = *reinterpret_cast<uint32_t*>(&q);
            }
            *reinterpret_cast<uint4*>(s_act + tile_off(f0 + c * 8, lt)) = u;
          }
          umma::fence_proxy_async();
        } else {
#pragma unroll
          for (int j = 0; j < W; ++j) {
            if (h[j] > 0.f) maskH |= 1ull << j;
            h[j] = __half2float(__float2half_rn(fmaxf(h[j], 0.f)));
          }
        }
        umma::fence_before_sync();
        umma::bar_sync(1, kTile);
      }
      if (!go) break;

      {
        // -- output, loss, dL/dy (scaled by S)
        float y = 0.f;
#pragma unroll
        for (int j = 0; j < W; ++j) y += h[j] * s_wout[j];
        float dy = 0.f;
        if (valid && p.ext_dy) {
          dy = p.ext_dy[i] * S;
          if (!isfinite(y)) atomicOr(&md.st->overflow, 1u);
        } else if (valid) {
          const float d = y - target;
          if (p.loss == DVNR_LOSS_L1) {
            loss_acc += fabsf(d);
            dy = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * (S * p.inv_batch);
          } else {
            loss_acc += d * d;
            dy = 2.f * d * (S * p.inv_batch);
          }
          if (!isfinite(y)) atomicOr(&md.st->overflow, 1u);
          if (p.dbg_y && cur == 0) {
            p.dbg_y[i] = y;
            p.dbg_tgt[i] = target;
            const uint32_t* crd = s_crd + 3 * (b * kTile + lt);
            p.dbg_coords[3 * i] = crd[0];
            p.dbg_coords[3 * i + 1] = crd[1];
            p.dbg_coords[3 * i + 2] = crd[2];
          }
        }
        // dW_out += fp16(dy) h_H, reduced over the warp (reduce-scatter)
        {
          const float dy16 = __half2float(__float2half_rn(dy));
          float v[W];
#pragma unroll
          for (int j = 0; j < W; ++j) v[j] = dy16 * h[j];
          int n = W;
#pragma unroll
          for (int s = 16; s >= 1; s >>= 1) {
            if (n > 1) {
              const bool upper = (lane & s) != 0;
              const int half = n / 2;
#pragma unroll
              for (int j = 0; j < W / 2; ++j) {
                if (j < half) {
                  const float send = upper ? v[j] : v[j + half];
                  const float keep = upper ? v[j + half] : v[j];
                  v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
                }
              }
              n = half;
            } else {
              v[0] += __shfl_xor_sync(0xffffffffu, v[0], s);
            }
          }
#pragma unroll
          for (int j = 0; j < NOUT; ++j) acc_out[j] += v[j];
        }
        // dZ_H = fp16(dy w_out) where z_H > 0
        const uint32_t f0 = (uint32_t)(H - 1) * W;
#pragma unroll
        for (int c = 0; c < W / 8; ++c) {
          uint4 u;
          uint32_t* pu = &u.x;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int a = c * 8 + 2 * j;
            const float v0 = ((maskH >> a) & 1ull) ? dy * s_wout[a] : 0.f;
            const float v1 = ((maskH >> (a + 1)) & 1ull) ? dy * s_wout[a + 1] : 0.f;
            __half2 q = __floats2half2_rn(v0, v1);
            pu[j] = *reinterpret_cast<uint32_t*>(&q);
          }
          *reinterpret_cast<uint4*>(s_dz + tile_off(f0 + c * 8, lt)) = u;
        }
      }
      umma::fence_proxy_async();
      umma::fence_before_sync();
      umma::bar_sync(1, kTile);

      // -- backward through layers H .. 2: layer k maps H_{k-1} -> Z_k with W_{k-1}
      for (int k = H; k >= 2; --k) {
        if (lt == 0) {
          umma::fence_after_sync();
          const uint32_t dz0 = umma::smem_u32(s_dz) + ((uint32_t)((k - 1) * W) >> 3) * 2048u;
          const uint32_t act0 = umma::smem_u32(s_act) + (p.lay.act_off[k - 1] >> 3) * 2048u;
          // dW_{k-1} += dZ_k^T H_{k-1} (K = samples; both operands MN-major)
          const uint32_t idw = umma::idesc_f16(kTile, W, 1, 1);
          for (int ks = 0; ks < kTile / 16; ++ks) {
            const uint64_t a = umma::sdesc(dz0 + ks * 256u, 128u, 2048u);
            const uint64_t bb = umma::sdesc(act0 + ks * 256u, 128u, 2048u);
            umma::mma_f16(tmem + p.lay.dw_col[k - 1], a, bb, idw, (first_tile && ks == 0) ? 0u : 1u);
          }
          // dH_{k-1} = dZ_k W_{k-1} (A K-major over the W outputs, B MN-major)
          const uint32_t ibw = umma::idesc_f16(kTile, W, 0, 1);
          const uint32_t w0 = umma::smem_u32(smem + p.lay.smem_w + p.lay.wbyte[k - 1]);
          const uint32_t wb = (uint32_t)(W >> 3) * 128u;
          for (int kk = 0; kk < W / 16; ++kk) {
            const uint64_t a = umma::sdesc(dz0 + kk * 4096u, 2048u, 128u);
            const uint64_t bb = umma::sdesc(w0 + kk * 256u, 128u, wb);
            umma::mma_f16(tmem, a, bb, ibw, kk > 0);
          }
          umma::commit(mbar);
        }
        if (!mma_wait()) {
          go = false;
          break;
        }
        umma::fence_after_sync();
        float dh[W];
#pragma unroll
        for (int c = 0; c < W / 16; ++c) {
          float v[16];
          umma::ld16(tl + c * 16, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) dh[c * 16 + j] = v[j];
        }
        umma::ld_wait();
        const uint32_t fa = p.lay.act_off[k - 1], fz = (uint32_t)(k - 2) * W;
#pragma unroll
        for (int c = 0; c < W / 8; ++c) {
          const uint4 hv = *reinterpret_cast<const uint4*>(s_act + tile_off(fa + c * 8, lt));
          const uint32_t* ph = &hv.x;
          uint4 u;
          uint32_t* pu = &u.x;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __half2 hh = *reinterpret_cast<const __half2*>(ph + j);
            const float2 hf = __half22float2(hh);
            const float v0 = hf.x > 0.f ? dh[c * 8 + 2 * j] : 0.f;
            const float v1 = hf.y > 0.f ? dh[c * 8 + 2 * j + 1] : 0.f;
            __half2 q = __floats2half2_rn(v0, v1);
            pu[j] = *reinterpret_cast<uint32_t*>(&q);
          }
          *reinterpret_cast<uint4*>(s_dz + tile_off(fz + c * 8, lt)) = u;
        }
        umma::fence_proxy_async();
        umma::fence_before_sync();
        umma::bar_sync(1, kTile);
      }
      if (!go) break;
      // -- layer 1: dW_0 += dZ_1^T X0 and dL/dX0 = dZ_1 W_0 into slot b's
      // columns, once slot b's gathering group has read the slot's previous
      // dL/dX0; the commit on dx[b] hands both the gradient and the free X0
      // slot to that group (no wait here: the next tile's products queue
      // behind these in the tensor core)
      if (lt == 0) {
        bool ok = true;
        if (t >= 2) ok = umma::mbar_wait_bounded(dxfree + b, (use - 1u) & 1u, abort_flag, kWaitCycles);
        if (ok) {
          umma::fence_after_sync();
          const uint32_t dz0 = umma::smem_u32(s_dz);
          const int in = (int)p.lay.dpad;  // layer 0's K includes the zero padding
          const uint32_t idw = umma::idesc_f16(kTile, in, 1, 1);
          for (int ks = 0; ks < kTile / 16; ++ks) {
            const uint64_t a = umma::sdesc(dz0 + ks * 256u, 128u, 2048u);
            const uint64_t bb = umma::sdesc(x0 + ks * 256u, 128u, 2048u);
            umma::mma_f16(tmem + p.lay.dw_col[0], a, bb, idw, (first_tile && ks == 0) ? 0u : 1u);
          }
          const uint32_t ibw = umma::idesc_f16(kTile, in, 0, 1);
          const uint32_t w0 = umma::smem_u32(smem + p.lay.smem_w + p.lay.wbyte[0]);
          const uint32_t wb = (uint32_t)(W >> 3) * 128u;
          for (int kk = 0; kk < W / 16; ++kk) {
            const uint64_t a = umma::sdesc(dz0 + kk * 4096u, 2048u, 128u);
            const uint64_t bb = umma::sdesc(w0 + kk * 256u, 128u, wb);
            umma::mma_f16(tmem + p.lay.dx_col[b], a, bb, ibw, kk > 0);
          }
          umma::commit(dxr + b);
        }
      }
      first_tile = false;
      ++t;
    }
    // the last tile's products complete before the run's dW leave TMEM
    if (go && cur >= 0 && t > 0) {
      if (group_wait(dxr + ((t - 1) & 1), (uint32_t)((t - 1) >> 1) & 1u)) flush();
    }
  } else {
    // -------------------------------------------------- gathering warps --
    // group gj (warps 4 + 4 gj .. 7 + 4 gj) takes the tiles t = gj, gj + 2,
    // ... through X0 slot gj and its own staging area
    const int gj = (warp >> 2) - 1;
    const uint32_t bar_id = 2u + (uint32_t)gj;
    uint8_t* stage = smem + p.lay.smem_stage + (uint32_t)gj * (uint32_t)p.lay.stage_levels * kStageLevelBytes;
    auto group_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      umma::mbar_wait_bounded(bar, parity, abort_flag, kWaitCycles);
      return !umma::bar_or(bar_id, kTile, *abort_flag != 0u);
    };
    // sample, target and encoding of tile g into slot b, then the slot's arrival
    auto gather = [&](int64_t g, int b) -> uint3 {
      int tile;
      const int model = model_of(g, tile);
      const MpModel mg = p.models[model];
      SampleParams sp;
      sp.key = p.key;
      sp.n_bnd = p.n_bnd;
      sp.qtab = p.qtab;
      sp.model = mg.slot;
      const uint32_t iter = p.explicit_iter ? p.iter : mg.st->iter;
      const int i = tile * kTile + lt;
      const bool valid = i < p.batch;
      uint3 mc = make_uint3(0u, 0u, 0u);
      if (valid)
        mc = p.ext_coords ? make_uint3(p.ext_coords[3 * i], p.ext_coords[3 * i + 1], p.ext_coords[3 * i + 2])
                          : draw_sample(sp, (uint32_t)i, iter);
      VolCorners vc{};
      if (valid && mg.vol) vc = vol_fetch(mg.vol, mg.nx, mg.ny, mg.nz, mc);  // in flight during the encode
      encode_to_tile_staged(p.lv, mg.theta16, mc, valid, smem + p.lay.smem_x0[b], (uint32_t)lt, stage,
                            p.lay.stage_levels, nullptr, 0);
      float vmin, inv_range;
      value_range(mg.st, vmin, inv_range);
      s_tgt[b * kTile + lt] = (valid && mg.vol) ? (vol_interp(vc) - vmin) * inv_range : 0.f;
      uint32_t* crd = s_crd + 3 * (b * kTile + lt);
      crd[0] = mc.x;
      crd[1] = mc.y;
      crd[2] = mc.z;
      umma::fence_proxy_async();
      umma::mbar_arrive(full + b);
      return mc;
    };
    int wv = p.wave_first - 1;
    int64_t g = 0, ge = 0, t = 0;
    while (next_tile(wv, g, ge)) {
      if ((int)(t & 1) != gj) {  // the other group's tile
        ++t;
        continue;
      }
      const int b = gj;
      const uint3 mc = gather(g, b);
      // tile t's dL/dX0 (its products complete, and with them every read of
      // X0 slot b), read back 16 columns at a time and reduced into the
      // table gradients
      if (!group_wait(dxr + b, (uint32_t)(t >> 1) & 1u)) break;
      umma::fence_after_sync();
      int tile;
      const int model = model_of(g, tile);
      if (lt == 0) mem_model[gj] = model;
      const MpModel ms = p.models[model];
      const int i = tile * kTile + lt;
      const bool valid = i < p.batch;
      const float inv_S = 1.0f / scale_of(ms);
      float* dbg_row = (p.dbg_dx0 && model == 0 && valid) ? p.dbg_dx0 + (size_t)i * D : nullptr;
      bool bad = false;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c * 16 >= D) break;
        float d[16];
        umma::ld16(tl + p.lay.dx_col[b] + (uint32_t)(c * 16), d);
        umma::ld_wait();
        if (!valid) continue;
        if (dbg_row) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c * 16 + j < D) dbg_row[c * 16 + j] = d[j] * inv_S;
        }
        if (c * 16 + 16 <= D)
          bad |= scatter_chunk<F, false>(p.lv, ms.grad, mc, d, c * 16);
        else
          bad |= scatter_chunk<F, true>(p.lv, ms.grad, mc, d, c * 16);
      }
      if (bad) atomicOr(&ms.st->overflow, 1u);
      // slot b's dL/dX0 has been read: the chain may overwrite it
      umma::fence_before_sync();
      umma::mbar_arrive(dxfree + b);
      umma::bar_sync(bar_id, kTile);
      if (lt == 0) mem_model[gj] = -1;
      ++t;
    }
  }

  // -- teardown (both groups have left their loops)
  umma::fence_before_sync();
  __syncthreads();
  if (*abort_flag && tid == 0) {
    // every product this thread issued completes (bounded) before TMEM is freed
    umma::commit(fin);
    const long long t0 = clock64();
    while (!umma::mbar_try_wait(fin, 0u) && clock64() - t0 < kWaitCycles) {
    }
    // the steps of the models whose gradients are incomplete: count the
    // timeout and have Adam skip them (kStepAborted clears the gradient)
    if (cur >= 0) {
      atomicAdd(&md.st->timeouts, 1u);
      atomicOr(&md.st->overflow, kStepAborted);
    }
    for (int j = 0; j < 2; ++j) {
      const int mm = mem_model[j];
      if (mm >= 0 && mm != cur && (j == 0 || mm != mem_model[0])) {
        const MpModel mx = p.models[mm];
        atomicAdd(&mx.st->timeouts, 1u);
        atomicOr(&mx.st->overflow, kStepAborted);
      }
    }
  }
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, p.lay.tmem_cols);
}

// The step's active models in index order (a block-wide exclusive scan of
// model_active over the models): sched[0] = count, sched[1 + a] = index of the
// a-th active model, sched[1 + n + m] = position of model m or -1. One block
// of 1024 threads; launched before every grouped training step.
__global__ void __launch_bounds__(1024) k_mp_schedule(const MpModel* __restrict__ models, int n,
                                                      int32_t* __restrict__ sched) {
  __shared__ int s_cnt[32];
  __shared__ int s_total;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int base = 0;
  for (int c = 0; c < n; c += blockDim.x) {
    const int m = c + tid;
    const bool act = m < n && model_active(models[m].st);
    const uint32_t b = __ballot_sync(0xffffffffu, act);
    if (lane == 0) s_cnt[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
      const int v = lane < nw ? s_cnt[lane] : 0;
      int x = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane < nw) s_cnt[lane] = x - v;  // exclusive prefix of the warps
      if (lane == 31) s_total = x;
    }
    __syncthreads();
    const int pos = base + s_cnt[warp] + __popc(b & ((1u << lane) - 1u));
    if (m < n) {
      sched[1 + n + m] = act ? pos : -1;
      if (act) sched[1 + pos] = m;
    }
    base += s_total;
    __syncthreads();
  }
  if (tid == 0) sched[0] = base;
}

// Loop control of the early-stop training graph, which runs the steps of a
// call as a conditional WHILE node whose body is a fixed number of steps
// followed by this kernel. It sets the node's condition for the next body
// run: some model of the group is still active (budget left, moving average
// above the threshold) and fewer body runs than the call allows have been
// made. arm >= 0 (the node in front of the loop) starts the run count at arm;
// arm < 0 (the body's last node) continues it. Each granted run adds the
// body's kernel count to the pinned host word `launches` (may be null).
__global__ void __launch_bounds__(256) k_mp_continue(const MpModel* __restrict__ models, int n,
                                                     int32_t* __restrict__ runs_left, int32_t arm,
                                                     unsigned long long* launches, int32_t body_launches,
                                                     cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) any |= model_active(models[m].st) ? 1 : 0;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int32_t r = arm >= 0 ? arm : *runs_left;
    const bool go = any != 0 && r > 0;
    *runs_left = go ? r - 1 : 0;
    if (go && launches) *launches += (unsigned long long)body_launches;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

// --------------------------------------------------------- decode kernel ---
template <int W, int F>
__global__ void __launch_bounds__(kTile, F <= 2 ? kDecodeCtasPerSm : 1) k_mp_decode(const __grid_constant__ MpDecodeParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 8);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(smem + 12);
  uint8_t* s_act = smem + p.lay.smem_act;
  const float* s_wout = reinterpret_cast<const float*>(smem + p.lay.smem_wout);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = p.D, H = p.H;
  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    *abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, p.lay.tmem_cols);
  load_weights(p.theta16, p.w_off, D, H, W, p.lay, smem);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  bool inflight = false;  // thread 0, as in k_mp_train
  long long wait_limit = p.first_wait_cycles;
  float vmin, inv_range;
  value_range(p.st, vmin, inv_range);
  const float range = inv_range > 0.f ? ordered_to_float(p.st->enc_max) - vmin : 0.f;

  for (int64_t t = blockIdx.x; t < p.n_tiles; t += gridDim.x) {
    const int64_t i = t * kTile + tid;
    const bool valid = i < p.n;
    uint3 m = make_uint3(0u, 0u, 0u);
    if (valid) {
      if (p.grid_mode == 2) {
        const int64_t k = (int64_t)fdiv((uint64_t)i, p.div_nr), ray = p.r0 + (i - k * p.nr);
        const int64_t ry = (int64_t)fdiv((uint64_t)ray, p.div_npx);
        const int px = p.rb.px0 + (int)(ray - ry * p.rb.npx), py = p.rb.py0 + (int)ry;
        m = make_uint3(dec_unit_to_fixed(frame_x(p.rf, px), p.rb.origin[0], p.rb.nstore[0]),
                       dec_unit_to_fixed(frame_y(p.rf, py), p.rb.origin[1], p.rb.nstore[1]),
                       dec_unit_to_fixed(frame_z(p.rf, p.rb.k0 + (int)k), p.rb.origin[2], p.rb.nstore[2]));
      } else if (p.grid_mode == 3) {
        m = make_uint3(p.coords[3 * i], p.coords[3 * i + 1], p.coords[3 * i + 2]);
      } else if (p.grid_mode) {
        const uint64_t q1 = fdiv((uint64_t)i, p.div_e0), q2 = fdiv(q1, p.div_e1);
        const uint64_t x = (uint64_t)i - q1 * (uint64_t)p.e[0], y = q1 - q2 * (uint64_t)p.e[1], z = q2;
        m = make_uint3(dec_grid_fixed(x + p.ghost, p.nstore[0], p.div_fix[0]),
                       dec_grid_fixed(y + p.ghost, p.nstore[1], p.div_fix[1]),
                       dec_grid_fixed(z + p.ghost, p.nstore[2], p.div_fix[2]));
      } else {
        m = make_uint3(dec_unit_to_fixed(p.xyz[3 * i], p.origin[0], p.nstore[0]),
                       dec_unit_to_fixed(p.xyz[3 * i + 1], p.origin[1], p.nstore[1]),
                       dec_unit_to_fixed(p.xyz[3 * i + 2], p.origin[2], p.nstore[2]));
      }
    }
    encode_to_tile<F, DVNR_DEC_PAIR, DVNR_DEC_GROUP, true>(p.lv, p.theta16, m, valid, s_act, (uint32_t)tid,
                                                           (int)p.lay.dpad);
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    // the epilogues take the layer's W outputs in chunks of CH columns, so
    // that few registers hold activations; the last one forms the output
    // y = sum_j fp16(relu(h_j)) w_j in order j = 0 .. W-1
    constexpr int CH = W >= 32 ? 32 : W;
    float y = 0.f;
    for (int k = 0; k < H; ++k) {
      if (tid == 0) {
        umma::fence_after_sync();
        issue_forward(tmem, smem, p.lay, k, k == 0 ? (int)p.lay.dpad : W, W);
        umma::commit(mbar);
        inflight = true;
      }
      if (umma::mbar_wait_bounded(mbar, phase, abort_flag, wait_limit)) inflight = false;
      wait_limit = kWaitCycles;
      phase ^= 1u;
      __syncthreads();
      if (*abort_flag) goto teardown;
      umma::fence_after_sync();
      const bool last = k == H - 1;
      const uint32_t f0 = last ? 0u : p.lay.act_off[k + 1];
#pragma unroll
      for (int c = 0; c < W / CH; ++c) {
        float h[CH];
#pragma unroll
        for (int u = 0; u < CH / 16; ++u) {
          float v[16];
          umma::ld16(tl + c * CH + u * 16, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) h[u * 16 + j] = v[j];
        }
        umma::ld_wait();
        // ReLU on the binary16 pairs: max(fp16(x), 0) is fp16(max(x, 0)) for
        // every x (a zero may change sign, which no sum or product here sees)
        const __half2 zero2 = __float2half2_rn(0.f);
        if (!last) {
#pragma unroll
          for (int g = 0; g < CH / 8; ++g) {
            uint4 u;
            uint32_t* pu = &u.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              __half2 q = __hmax2(__floats2half2_rn(h[g * 8 + 2 * j], h[g * 8 + 2 * j + 1]), zero2);
              pu[j] = *reinterpret_cast<uint32_t*>(&q);
            }
            *reinterpret_cast<uint4*>(s_act + tile_off(f0 + c * CH + g * 8, tid)) = u;
          }
        } else {
#pragma unroll
          for (int j = 0; j < CH; j += 2) {
            const float2 r = __half22float2(__hmax2(__floats2half2_rn(h[j], h[j + 1]), zero2));
            y += r.x * s_wout[c * CH + j];
            y += r.y * s_wout[c * CH + j + 1];
          }
        }
      }
      if (!last) umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
    }
    if (valid) p.out[i] = p.grid_mode == 3 ? y : y * range + vmin;
  }
teardown:
  if (*abort_flag && tid == 0) {
    if (inflight) {  // the MMA of the phase before `phase`
      const long long t0 = clock64();
      while (!umma::mbar_try_wait(mbar, phase ^ 1u) && clock64() - t0 < kWaitCycles) {
      }
    }
    atomicAdd(const_cast<uint32_t*>(&p.st->timeouts), 1u);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, p.lay.tmem_cols);
}

// ------------------------------------------------------ UMMA self-test -----
// One 128 x 64 x 64 product per operand-major combination on small integers
// divided by powers of two (exact in FP16 and FP32), against a SIMT product.
__global__ void __launch_bounds__(128) k_umma_selftest(int32_t* mismatches) {
  __shared__ __align__(1024) uint8_t sa[128 * 64 * 2];
  __shared__ __align__(1024) uint8_t sb[64 * 64 * 2];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ uint32_t abort_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  auto Aval = [](int m, int k) { return (float)(((m * 3 + k * 5) % 17) - 8) * 0.125f; };
  auto Bval = [](int k, int n) { return (float)(((k * 7 + n * 11) % 13) - 6) * 0.25f; };
  if (tid == 0) {
    umma::mbar_init(&bar, 1);
    abort_s = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) umma::tmem_alloc(&tslot, 64);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tslot;
  uint32_t phase = 0;
  bool inflight = false;  // thread 0: committed, completion not yet seen
  for (int cs = 0; cs < 4; ++cs) {
    const int a_mn = cs & 1, b_mn = cs >> 1;
    // A: M = 128, K = 64. K-major: core (m/8, k/8) at ((k/8)*16 + m/8)*128,
    // 16-byte rows along K. MN-major: core at ((m/8)*8 + k/8)*128, rows along M.
    for (int e = tid; e < 128 * 64; e += 128) {
      const int m = e / 64, k = e % 64;
      uint32_t off;
      if (!a_mn)
        off = ((((k >> 3) << 4) + (m >> 3)) << 7) + ((m & 7) << 4) + ((k & 7) << 1);
      else
        off = ((((m >> 3) << 3) + (k >> 3)) << 7) + ((k & 7) << 4) + ((m & 7) << 1);
      *reinterpret_cast<__half*>(sa + off) = __float2half_rn(Aval(m, k));
    }
    // B: K = 64, N = 64. K-major: core at ((k/8)*8 + n/8)*128 rows along K;
    // MN-major: core at ((n/8)*8 + k/8)*128 rows along N.
    for (int e = tid; e < 64 * 64; e += 128) {
      const int k = e / 64, n = e % 64;
      uint32_t off;
      if (!b_mn)
        off = ((((k >> 3) << 3) + (n >> 3)) << 7) + ((n & 7) << 4) + ((k & 7) << 1);
      else
        off = ((((n >> 3) << 3) + (k >> 3)) << 7) + ((k & 7) << 4) + ((n & 7) << 1);
      *reinterpret_cast<__half*>(sb + off) = __float2half_rn(Bval(k, n));
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
      const uint32_t a0 = umma::smem_u32(sa), b0 = umma::smem_u32(sb);
      const uint32_t id = umma::idesc_f16(128, 64, a_mn, b_mn);
      for (int kk = 0; kk < 4; ++kk) {
        uint64_t a, b;
        if (!a_mn) a = umma::sdesc(a0 + kk * 2 * 2048, 2048, 128);   // LBO along K, SBO along M
        else a = umma::sdesc(a0 + kk * 2 * 128, 128, 1024);          // LBO along K, SBO along M
        if (!b_mn) b = umma::sdesc(b0 + kk * 2 * 1024, 1024, 128);
        else b = umma::sdesc(b0 + kk * 2 * 128, 128, 1024);
        umma::mma_f16(tmem, a, b, id, kk > 0);
      }
      umma::commit(&bar);
      inflight = true;
    }
    if (umma::mbar_wait_bounded(&bar, phase, &abort_s, kWaitCycles)) inflight = false;
    phase ^= 1u;
    __syncthreads();
    if (abort_s) break;
    umma::fence_after_sync();
    int bad = 0;
    const int m = tid;
    for (int c = 0; c < 4; ++c) {
      float v[16];
      umma::ld16(tmem + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      umma::ld_wait();
      for (int j = 0; j < 16; ++j) {
        const int n = c * 16 + j;
        float ref = 0.f;
        for (int k = 0; k < 64; ++k) ref += Aval(m, k) * Bval(k, n);
        bad += v[j] != ref;
      }
    }
    atomicAdd(mismatches + cs, bad);
    umma::fence_before_sync();
    __syncthreads();
  }
  if (abort_s && tid == 0) {
    mismatches[4] = 1;
    if (inflight) {  // let the product of the phase before `phase` finish before TMEM is freed
      const long long t0 = clock64();
      while (!umma::mbar_try_wait(&bar, phase ^ 1u) && clock64() - t0 < kWaitCycles) {
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, 64);
}

// ----------------------------------------------------------- host side -----
template <int W, int F>
void set_smem_attr(bool train, uint32_t bytes) {
  // the largest shared-memory carveout: these kernels hold big tiles in
  // shared memory, and with no preference the occupancy query assumes a
  // partition that fits one CTA per SM
  if (train) {
    cudaFuncSetAttribute(k_mp_train<W, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_mp_train<W, F>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    if constexpr (F == 2) {
      cudaFuncSetAttribute(k_mp_train_ws<W, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_mp_train_ws<W, F>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
    }
  } else {
    cudaFuncSetAttribute(k_mp_decode<W, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_mp_decode<W, F>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
  }
}

template <int W, int F>
void launch_train_wf(const MpParams& p, int grid, cudaStream_t s) {
  if constexpr (F == 2) {
    if (p.lay.ws) {
      count_train_launch(true);
      k_mp_train_ws<W, F><<<grid, 3 * kTile, p.lay.smem_bytes, s>>>(p);
      return;
    }
  }
  count_train_launch(false);
  k_mp_train<W, F><<<grid, kTile, p.lay.smem_bytes, s>>>(p);
}
template <int W, int F>
void launch_decode_wf(const MpDecodeParams& p, cudaStream_t s) {
  // one full wave of resident CTAs (registers can hold fewer per SM than
  // shared and tensor memory allow)
  const int per_sm = resident_ctas(k_mp_decode<W, F>, kTile, p.lay.smem_bytes, p.lay.ctas_per_sm);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(p.n_tiles, (int64_t)sm_count() * per_sm));
  k_mp_decode<W, F><<<grid, kTile, p.lay.smem_bytes, s>>>(p);
}


// Per-model cache of the FP16 path: device tables of the last grouped call
// and its captured CUDA graph.
struct MpCache {
  std::vector<uint64_t> uids;  // dvnr_model_s::uid of each model of the cached call
  std::vector<const float*> vols;
  std::vector<uint32_t> slots;
  dvnr_train_cfg cfg{};
  int graph_steps = 0;
  // fixed graphs of 2^k steps (k = kMinGraphLog .. kMaxGraphLog), captured on
  // first use: a call of n steps replays the binary digits of n
  cudaGraphExec_t fixed_exec[kMaxGraphLog + 1] = {};
  cudaGraph_t fixed_graph[kMaxGraphLog + 1] = {};
  MpModel* d_models = nullptr;
  AdamModelPtrs* d_adam = nullptr;
  int32_t* d_sched = nullptr;  // active-model schedule, 1 + 2 n ints, then the loop's run count
  cudaGraphExec_t exec = nullptr;  // the early-stop loop graph
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  int64_t wave_tiles = 0;
  int ctas_per_sm = 0;
  bool scheduled = false;  // the captured graph launches k_mp_schedule
  bool interleaved = false;  // the captured steps interleave Adam per wave
  bool ws = false;           // the captured steps launch k_mp_train_ws
  // early-stop graph: arm node -> WHILE { steps, k_mp_continue }
  bool looped = false;          // exec holds the loop graph
  bool loop_unavailable = false;  // building it failed once: fixed graphs only
  cudaGraphNode_t arm_node = nullptr;
  cudaKernelNodeParams arm_params{};
  void* arm_args[7] = {};
  const MpModel* arm_models = nullptr;
  int arm_n = 0;
  int32_t* arm_runs = nullptr;
  int32_t arm_value = 0;
  unsigned long long* arm_launches = nullptr;  // host word (device-mapped alias below)
  unsigned long long* arm_launches_dev = nullptr;
  int32_t arm_body = 0;
  cudaGraphConditionalHandle arm_cond = 0;
  bool any_graph() const {
    bool any = exec != nullptr;
    for (int k = 0; k <= kMaxGraphLog; ++k) any |= fixed_exec[k] != nullptr;
    return any;
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    for (int k = 0; k <= kMaxGraphLog; ++k) {
      if (fixed_exec[k]) cudaGraphExecDestroy(fixed_exec[k]);
      if (fixed_graph[k]) cudaGraphDestroy(fixed_graph[k]);
      fixed_exec[k] = nullptr;
      fixed_graph[k] = nullptr;
    }
    arm_node = nullptr;
    looped = false;
    graph_steps = 0;
  }
  void clear() {
    // a graph of an earlier call may still run on another stream, writing
    // the launch counter and reading the descriptor tables
    if (any_graph() || arm_launches || d_models) cudaDeviceSynchronize();
    drop_graph();
    device_counter_free(arm_launches);
    arm_launches = nullptr;
    arm_launches_dev = nullptr;
    if (d_models) dev_free(d_models);
    if (d_adam) dev_free(d_adam);
    if (d_sched) dev_free(d_sched);
    if (cap) cudaStreamDestroy(cap);
    d_models = nullptr;
    d_adam = nullptr;
    d_sched = nullptr;
    cap = nullptr;
    uids.clear();
    vols.clear();
    slots.clear();
    graph_steps = 0;
  }
};

bool same_cfg(const dvnr_train_cfg& a, const dvnr_train_cfg& b) {
  return a.lr == b.lr && a.beta1 == b.beta1 && a.beta2 == b.beta2 && a.eps == b.eps &&
         a.weight_decay == b.weight_decay && a.lambda_bnd == b.lambda_bnd &&
         a.sigma_bnd == b.sigma_bnd && a.batch == b.batch && a.loss == b.loss &&
         a.growth_interval == b.growth_interval && a.seed == b.seed &&
         a.stop_loss == b.stop_loss && a.stop_decay == b.stop_decay;
}

MpParams base_params(const dvnr_model m, const MpLayout& lay, const dvnr_train_cfg* cfg) {
  MpParams p{};
  p.lv = m->lv;
  p.D = m->lv.in_dim;
  p.H = m->mlp.n_hidden;
  for (int k = 0; k <= m->mlp.n_hidden; ++k) p.w_off[k] = m->w_off[k];
  p.lay = lay;
  p.batch = cfg->batch;
  p.n_bnd = (int32_t)std::floor((double)cfg->lambda_bnd * (double)cfg->batch);
  p.loss = cfg->loss;
  p.tiles_per_model = (cfg->batch + kTile - 1) / kTile;
  p.key = make_uint2((uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32));
  p.qtab = m->qtab;
  p.inv_batch = 1.0f / (float)cfg->batch;
  p.first_wait_cycles = g_first_wait.load();
  p.wave_first = 0;
  p.wave_end = -1;
  return p;
}

int train_grid(const MpParams& p) {
  const int64_t cap = (int64_t)sm_count() * p.lay.ctas_per_sm;
  return (int)std::max<int64_t>(1, std::min<int64_t>(p.total_tiles, cap));
}

// Wave schedule: a wave holds about as many models as fit their FP16 tables
// and FP32 gradients into a quarter of the L2, but at least enough tiles
// for half a tile per CTA; the autotuner also tries waves of whole grid
// rounds (k tiles per CTA, which keep every CTA busy when models are small)
// and a single wave. DVNR_WAVE_MODELS=v fixes waves of v models,
// DVNR_WAVE_TILES=v waves of v tiles.
int heuristic_models_per_wave(const MpParams& p, const dvnr_model m, int n_models) {
  int l2 = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (l2 <= 0) l2 = 64 << 20;
  const double per_model = (double)m->n_params * 6.0;
  const int by_cache = (int)std::max(1.0, std::floor(0.25 * (double)l2 / per_model));
  const int64_t G0 = train_grid(p);
  const int by_occupancy = (int)((G0 + 2 * p.tiles_per_model - 1) / (2 * p.tiles_per_model));
  return std::min(std::max(by_cache, by_occupancy), n_models);
}

void set_wave_tiles(MpParams& p, int64_t tiles) {
  p.wave_tiles = std::max<int64_t>(1, std::min<int64_t>(tiles, p.total_tiles));
}

void set_waves(MpParams& p, const dvnr_model m, int n_models) {
  int mw = heuristic_models_per_wave(p, m, n_models);
  if (const char* e = getenv("DVNR_WAVE_MODELS")) {
    const int v = atoi(e);
    if (v > 0) mw = v;
  }
  int64_t tiles = (int64_t)mw * p.tiles_per_model;
  if (const char* e = getenv("DVNR_WAVE_TILES")) {  // waves of v tiles (may split models)
    const long long v = atoll(e);
    if (v > 0) tiles = v;
  }
  set_wave_tiles(p, tiles);
}

dvnr_status launch_train(const MpParams& p, int W, int F, int n_models, cudaStream_t s) {
  if (p.sched) {
    ProfScope ps("mp_schedule", s);
    k_mp_schedule<<<1, 1024, 0, s>>>(p.models, n_models, const_cast<int32_t*>(p.sched));
    DVNR_CUDA(cudaGetLastError());
  }
  {
    ProfScope ps("train_fused_fp16", s);
    DVNR_WF_DISPATCH(W, F, launch_train_wf, p, train_grid(p), s);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

// A step run wave by wave ("interleaved"): before the training launch of
// each wave, the Adam update of the models whose first tile lies in that
// wave (from the previous step's gradients), so that the FP16 tables the
// update writes and the gradients it clears are still in L2 when the wave
// gathers and scatters into them. Each model is updated before any of its
// tiles trains (launch order), and after all tiles of the previous step;
// the first step of a call trains without an update and the call ends with
// one update of every model, so the sequence of operations per model is that
// of the plain step (train, then Adam). Used when every model takes part in
// every step (no schedule).
dvnr_status launch_interleaved_step(const MpParams& q, int W, int F, int n, const AdamModelPtrs* d_adam,
                                    int64_t n_store, const AdamHyper& h, cudaStream_t s) {
  const int64_t T = q.total_tiles, wt = q.wave_tiles, tpm = q.tiles_per_model;
  const int n_waves = (int)((T + wt - 1) / wt);
  for (int w = 0; w < n_waves; ++w) {
    const int64_t t0 = (int64_t)w * wt, t1 = std::min(T, t0 + wt);
    const int m0 = (int)((t0 + tpm - 1) / tpm), m1 = (int)std::min<int64_t>(n, (t1 + tpm - 1) / tpm);
    if (m1 > m0) {
      dvnr_status rc = launch_adam(d_adam + m0, m1 - m0, n_store, h, s);
      if (rc != DVNR_OK) return rc;
    }
    MpParams pw = q;
    pw.wave_first = w;
    pw.wave_end = w + 1;
    dvnr_status rc = launch_train(pw, W, F, n, s);
    if (rc != DVNR_OK) return rc;
  }
  return DVNR_OK;
}

// Kernel launches of one interleaved step (for the launch count).
int64_t interleaved_launches(const MpParams& q, int n) {
  const int64_t T = q.total_tiles, wt = q.wave_tiles, tpm = q.tiles_per_model;
  const int n_waves = (int)((T + wt - 1) / wt);
  int64_t c = 0;
  for (int w = 0; w < n_waves; ++w) {
    const int64_t t0 = (int64_t)w * wt, t1 = std::min(T, t0 + wt);
    const int m0 = (int)((t0 + tpm - 1) / tpm), m1 = (int)std::min<int64_t>(n, (t1 + tpm - 1) / tpm);
    c += 1 + (m1 > m0 ? 1 : 0);
  }
  return c;
}

// Launch-shape autotuner of the grouped training step: on the first call
// for a configuration (encoding, MLP, batch, number of models) it times a
// whole step for each candidate -- CTAs per SM (as many as fit, or one),
// models per wave (the heuristic, half, double) or grid rounds per wave --
// in the step's layout (training launch then Adam; interleaved per wave
// with DVNR_INTERLEAVE=1) on the call's own models and volumes, with Adam
// in its dry mode (the same traffic, values written back unchanged), then
// clears what the trials wrote (weight gradients, loss sums, overflow flags;
// parameters, moments and step counters are not touched) and caches the
// fastest choice for the process. DVNR_AUTOTUNE=0 keeps the heuristic;
// DVNR_WAVE_MODELS fixes the wave size.
struct TuneChoice {
  int ctas_per_sm;
  int64_t wave_tiles;
  bool interleaved;
  bool ws;  // the warp-specialised kernel (k_mp_train_ws)
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;

// DVNR_TRAIN_WS: 1 selects k_mp_train_ws wherever its layout fits (unset: -1,
// and 0: k_mp_train).
int train_ws_env() {
  const char* e = getenv("DVNR_TRAIN_WS");
  if (!e) return -1;
  return atoi(e) != 0 ? 1 : 0;
}

std::string tune_key(const dvnr_model m, int n, const dvnr_train_cfg* cfg) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d:%.9g:%d:%d:%d:%d:%d", m->enc.n_levels, m->enc.n_features,
           m->enc.log2_T, m->enc.base_res, m->mlp.width, m->enc.growth, m->mlp.n_hidden, cfg->batch, n,
           cfg->lambda_bnd > 0.f ? 1 : 0, cfg->loss);
  return buf;
}

dvnr_status autotune(MpParams base, dvnr_model* models, int n, int W, int F, const AdamModelPtrs* d_adam,
                     const AdamHyper& h, int interleave_env, const MpLayout* lay_ws, bool only_ws,
                     TuneChoice* out, cudaStream_t s) {
  std::vector<TuneChoice> cands;
  auto add = [&](const MpParams& q, int ctas, bool ws) {
    const int hq = heuristic_models_per_wave(q, models[0], n);
    const int64_t G = train_grid(q), tpm = q.tiles_per_model, T = q.total_tiles;
    for (int64_t wt : {hq * tpm, std::max(1, hq / 2) * tpm, std::min(n, 2 * hq) * tpm, G, 2 * G, 4 * G, T}) {
      wt = std::max<int64_t>(1, std::min(wt, T));
      bool dup = false;
      for (const auto& c : cands) dup |= c.ctas_per_sm == ctas && c.wave_tiles == wt && c.ws == ws;
      if (dup) continue;
      // the interleaved layout is a candidate only when asked for
      // (DVNR_INTERLEAVE=1): measured slower on both workloads, its trials
      // would only lengthen the first call
      const bool il = interleave_env == 1 && !base.sched;  // needs every model in every step
      cands.push_back({ctas, wt, il, ws});
    }
  };
  if (!only_ws) {
    for (int ctas = base.lay.ctas_per_sm; ctas >= 1; ctas = ctas > 1 ? 1 : 0) {
      MpParams q = base;
      q.lay.ctas_per_sm = ctas;
      add(q, ctas, false);
      if (ctas == 1) break;
    }
  }
  if (lay_ws) {
    MpParams q = base;
    q.lay = *lay_ws;
    add(q, 1, true);
  }
  if (cands.empty()) cands.push_back({base.lay.ctas_per_sm, base.total_tiles, false, false});
  AdamHyper hd = h;
  hd.dry = 1;
  const int64_t n_store = models[0]->n_store;
  auto step = [&](const MpParams& q, bool il) -> dvnr_status {
    if (il) return launch_interleaved_step(q, W, F, n, d_adam, n_store, hd, s);
    dvnr_status rc = launch_train(q, W, F, n, s);
    if (rc != DVNR_OK) return rc;
    return launch_adam(d_adam, n, n_store, hd, s);
  };
  cudaEvent_t e0, e1;
  DVNR_CUDA(cudaEventCreate(&e0));
  DVNR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneChoice pick = cands[0];
  dvnr_status rc = DVNR_OK;
  for (const auto& c : cands) {
    MpParams q = base;
    if (c.ws) q.lay = *lay_ws;
    q.lay.ctas_per_sm = c.ctas_per_sm;
    set_wave_tiles(q, c.wave_tiles);
    if ((rc = step(q, c.interleaved)) != DVNR_OK) break;  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && rc == DVNR_OK; ++r) rc = step(q, c.interleaved);
    cudaEventRecord(e1, s);
    if (rc != DVNR_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = cuda_status(cudaGetLastError(), "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // undo the trial runs' side effects
  for (int i = 0; i < n; ++i) {
    dvnr_model m = models[i];
    DVNR_CUDA(cudaMemsetAsync(m->grad, 0, (size_t)m->n_store * sizeof(float), s));
    DVNR_CUDA(cudaMemsetAsync(&m->st->loss_sum, 0, sizeof(float), s));
    DVNR_CUDA(cudaMemsetAsync(&m->st->overflow, 0, sizeof(uint32_t), s));
  }
  if (rc != DVNR_OK) return rc;
  *out = pick;
  return DVNR_OK;
}

// The early-stop loop as one graph: an arm node (k_mp_continue with arm =
// the call's bound on body runs, set before every launch) in front of a
// conditional WHILE node whose body is G captured steps followed by
// k_mp_continue. The loop ends when no model of the group is active, so a
// group that stops early launches no further steps. DVNR_E_UNSUPPORTED when
// the runtime refuses a conditional-node call or pinned memory for the
// device-side launch count.
template <class Step>
dvnr_status build_loop_graph(MpCache* c, const MpModel* models, int n, int32_t* runs, int G, Step& one_step) {
  const dvnr_status no = DVNR_E_UNSUPPORTED;
  if (!c->arm_launches) {
    c->arm_launches = device_counter_new();
    c->arm_launches_dev = nullptr;
    if (c->arm_launches && cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->arm_launches_dev),
                                                    c->arm_launches, 0) != cudaSuccess)
      c->arm_launches_dev = nullptr;
  }
  if (!c->arm_launches_dev) return no;
  if (cudaGraphCreate(&c->graph, 0) != cudaSuccess) return no;
  cudaGraphConditionalHandle cond = 0;
  if (cudaGraphConditionalHandleCreate(&cond, c->graph, 0u, 0u) != cudaSuccess) return no;
  c->arm_models = models;
  c->arm_n = n;
  c->arm_runs = runs;
  c->arm_value = 0;
  c->arm_body = 3 * G + 1;  // schedule, train, Adam per step, then k_mp_continue
  c->arm_cond = cond;
  void* args[7] = {&c->arm_models, &c->arm_n, &c->arm_runs, &c->arm_value, &c->arm_launches_dev,
                   &c->arm_body, &c->arm_cond};
  for (int i = 0; i < 7; ++i) c->arm_args[i] = args[i];
  c->arm_params = cudaKernelNodeParams{};
  c->arm_params.func = reinterpret_cast<void*>(k_mp_continue);
  c->arm_params.gridDim = dim3(1, 1, 1);
  c->arm_params.blockDim = dim3(256, 1, 1);
  c->arm_params.sharedMemBytes = 0;
  c->arm_params.kernelParams = c->arm_args;
  c->arm_params.extra = nullptr;
  cudaGraphNode_t arm = nullptr, loop = nullptr;
  if (cudaGraphAddKernelNode(&arm, c->graph, nullptr, 0, &c->arm_params) != cudaSuccess) return no;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&loop, c->graph, &arm, nullptr, 1, &np) != cudaSuccess) return no;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  set_capturing(true);
  cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  dvnr_status rc = DVNR_OK;
  if (e == cudaSuccess) {
    for (int k = 0; k < G && rc == DVNR_OK; ++k) rc = one_step(c->cap);
    if (rc == DVNR_OK) {
      k_mp_continue<<<1, 256, 0, c->cap>>>(models, n, runs, -1, c->arm_launches_dev, c->arm_body, cond);
      e = cudaGetLastError();
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap, &out);
    if (e == cudaSuccess) e = e2;
  }
  set_capturing(false);
  if (rc != DVNR_OK) return rc;
  if (e != cudaSuccess) return no;
  if (cudaGraphInstantiate(&c->exec, c->graph, 0) != cudaSuccess) return no;
  c->arm_node = arm;
  c->graph_steps = G;
  c->looped = true;
  return DVNR_OK;
}

// `left` steps of a grouped call: directly while profiling or a lowered wait
// limit is active; else the early-stop loop graph when the call has a
// schedule, or the fixed graphs of 2^k steps (binary digits of `left`,
// k >= kMinGraphLog; the rest directly). step_launches: kernels per step.
template <class Step>
dvnr_status mp_train_steps(MpCache* c, const MpParams& p, int n, int64_t left, Step& one_step,
                           int64_t step_launches, cudaStream_t s) {
  // a lowered first-wait limit (failure-path tests) is not baked into graphs
  if (profiling_on() || p.first_wait_cycles != kWaitCycles) {
    count_eager_steps(left);
    for (int64_t i = 0; i < left; ++i) {
      dvnr_status rc = one_step(s);
      if (rc != DVNR_OK) return rc;
    }
    return DVNR_OK;
  }
  const int G = 1 << kMaxGraphLog;
  // models that can leave the group (budgets, stop rule) run under the
  // early-stop loop, which ends when none is left; the others, or a driver
  // without conditional nodes, replay fixed graphs (whose steps do nothing for
  // models that left). DVNR_GRAPH_LOOP=0 selects the fixed graphs for every
  // call.
  const char* gl = getenv("DVNR_GRAPH_LOOP");
  const bool want_loop = p.sched != nullptr && !c->loop_unavailable && !(gl && atoi(gl) == 0) && left >= 8;
  if (!c->cap) DVNR_CUDA(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (!c->exec && want_loop) {
    count_graph_capture();
    dvnr_status rc = build_loop_graph(c, p.models, n, c->d_sched + 1 + 2 * (size_t)n, G, one_step);
    if (rc != DVNR_OK) {
      // conditional nodes unavailable: keep the fixed graphs for this cache
      if (c->exec) cudaGraphExecDestroy(c->exec);
      if (c->graph) cudaGraphDestroy(c->graph);
      c->exec = nullptr;
      c->graph = nullptr;
      c->looped = false;
      c->loop_unavailable = true;
      cudaGetLastError();
      if (rc != DVNR_E_UNSUPPORTED) return rc;
    }
  }
  if (c->exec && want_loop) {
    // at most ceil(steps / G) body runs: every model's budget is at most
    // `steps`, and the step slots past a model's budget or stop are no-ops
    const int64_t runs = (left + G - 1) / G;
    c->arm_value = (int32_t)std::min<int64_t>(runs, 0x7FFFFFFF);
    DVNR_CUDA(cudaGraphExecKernelNodeSetParams(c->exec, c->arm_node, &c->arm_params));
    DVNR_CUDA(cudaGraphLaunch(c->exec, s));
    count_graph_replay();
    count_launches(1);  // the arm node; the body runs count themselves on the device
    return DVNR_OK;
  }
  // the graph of 2^k steps, captured on first use
  auto run_graph = [&](int k) -> dvnr_status {
    if (!c->fixed_exec[k]) {
      count_graph_capture();
      set_capturing(true);
      cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
      dvnr_status rc = DVNR_OK;
      if (e == cudaSuccess) {
        for (int g = 0; g < (1 << k) && rc == DVNR_OK; ++g) rc = one_step(c->cap);
        cudaError_t e2 = cudaStreamEndCapture(c->cap, &c->fixed_graph[k]);
        if (e == cudaSuccess) e = e2;
      }
      set_capturing(false);
      if (rc != DVNR_OK) return rc;
      DVNR_CUDA(e);
      DVNR_CUDA(cudaGraphInstantiate(&c->fixed_exec[k], c->fixed_graph[k], 0));
    }
    DVNR_CUDA(cudaGraphLaunch(c->fixed_exec[k], s));
    count_graph_replay();
    count_launches(step_launches << k);
    return DVNR_OK;
  };
  while (left >= G) {
    dvnr_status rc = run_graph(kMaxGraphLog);
    if (rc != DVNR_OK) return rc;
    left -= G;
  }
  for (int k = kMaxGraphLog - 1; k >= kMinGraphLog; --k) {
    if (left >= (1 << k)) {
      dvnr_status rc = run_graph(k);
      if (rc != DVNR_OK) return rc;
      left -= 1 << k;
    }
  }
  count_eager_steps(left);
  for (int64_t i = 0; i < left; ++i) {
    dvnr_status rc = one_step(s);
    if (rc != DVNR_OK) return rc;
  }
  return DVNR_OK;
}

}  // namespace

bool mp_supported(const dvnr_model m) {
  const int D = m->lv.in_dim, W = m->mlp.width, F = m->lv.F;
  if (!(W == 16 || W == 32 || W == 64)) return false;
  if (!(F == 1 || F == 2 || F == 4 || F == 8)) return false;
  if (D < 1 || D > 64) return false;  // padded with zeros to a multiple of 16 for layer 0
  MpLayout lay;
  return make_layout(m, true, lay) && make_layout(m, false, lay);
}

void mp_release(dvnr_model m) {
  if (m->mp) {
    MpCache* c = static_cast<MpCache*>(m->mp);
    c->clear();
    delete c;
    m->mp = nullptr;
  }
}

dvnr_status mp_train(dvnr_model* models, int n, const float* const* vols, const uint32_t* slots,
                     const dvnr_train_cfg* cfg, const AdamHyper& h, int64_t steps, bool uniform,
                     cudaStream_t s) {
  dvnr_model m0 = models[0];
  MpLayout lay;
  if (!make_layout(m0, true, lay)) {
    set_error("FP16 path: configuration exceeds shared or tensor memory");
    return DVNR_E_UNSUPPORTED;
  }
  if (!m0->mp) m0->mp = new MpCache();
  MpCache* c = static_cast<MpCache*>(m0->mp);
  bool hit = c->d_models && (int)c->uids.size() == n && same_cfg(c->cfg, *cfg);
  for (int i = 0; hit && i < n; ++i)
    hit = c->uids[i] == models[i]->uid && c->vols[i] == vols[i] && c->slots[i] == slots[i];
  if (!hit) {
    if (c->d_models) DVNR_CUDA(cudaStreamSynchronize(s));
    c->clear();
    std::vector<MpModel> hm((size_t)n);
    std::vector<AdamModelPtrs> ha((size_t)n);
    for (int i = 0; i < n; ++i) {
      dvnr_model m = models[i];
      hm[i] = MpModel{m->theta16, m->grad, vols[i], (int32_t)m->dims[0], (int32_t)m->dims[1],
                      (int32_t)m->dims[2], slots[i], m->st};
      ha[i] = AdamModelPtrs{m->theta, m->m1, m->m2, m->grad, m->theta16, m->st};
    }
    DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&c->d_models), sizeof(MpModel) * n));
    DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&c->d_adam), sizeof(AdamModelPtrs) * n));
    DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&c->d_sched), sizeof(int32_t) * (2 + 2 * (size_t)n)));
    DVNR_CUDA(cudaMemcpy(c->d_models, hm.data(), sizeof(MpModel) * n, cudaMemcpyHostToDevice));
    DVNR_CUDA(cudaMemcpy(c->d_adam, ha.data(), sizeof(AdamModelPtrs) * n, cudaMemcpyHostToDevice));
    c->uids.resize((size_t)n);
    for (int i = 0; i < n; ++i) c->uids[i] = models[i]->uid;
    c->vols.assign(vols, vols + n);
    c->slots.assign(slots, slots + n);
    c->cfg = *cfg;
  }
  MpParams p = base_params(m0, lay, cfg);
  p.total_tiles = (int64_t)p.tiles_per_model * n;
  p.n_models = n;
  // equal budgets and no stop rule: every model takes part in every step, so
  // the schedule is the identity and its kernel is left out
  p.sched = (uniform && cfg->stop_loss == 0.f) ? nullptr : c->d_sched;
  if (p.total_tiles * (int64_t)train_grid(p) >= (1LL << 32)) {
    set_error("FP16 path: %lld tiles per step is beyond the supported range", (long long)p.total_tiles);
    return DVNR_E_UNSUPPORTED;
  }
  p.models = c->d_models;
  // step layout: training launch then Adam, or interleaved per wave
  // (DVNR_INTERLEAVE=1; measured slower on both workloads)
  int interleave_env = -1;
  if (const char* e = getenv("DVNR_INTERLEAVE")) interleave_env = atoi(e) != 0 ? 1 : 0;
  bool interleaved = false;
  {
    const char* at = getenv("DVNR_AUTOTUNE");
    const bool tune = !(at && atoi(at) == 0) && !getenv("DVNR_WAVE_MODELS") && !getenv("DVNR_WAVE_TILES") &&
                      !profiling_on() && p.first_wait_cycles == kWaitCycles;
    // the warp-specialised kernel only when asked for (DVNR_TRAIN_WS=1),
    // where its layout fits: measured as fast as the plain kernel on the
    // 256^3 workload, not faster, its trials would only lengthen first calls
    const int ws_env = train_ws_env();
    MpLayout lay_ws;
    const bool ws_ok = ws_env == 1 && make_layout_ws(m0, lay_ws);
    const std::string key = tune_key(m0, n, cfg) + (p.sched ? ":s" : ":u") + ":ws" + std::to_string(ws_env);
    TuneChoice ch{0, 0, false, false};
    bool have = false;
    if (tune) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        ch = it->second;
        have = true;
      }
    }
    if (tune && !have) {
      const int W0 = m0->mlp.width, F0 = m0->lv.F;
      DVNR_WF_DISPATCH(W0, F0, set_smem_attr, true, lay.smem_bytes);
      dvnr_status rc = autotune(p, models, n, W0, F0, c->d_adam, h, interleave_env, ws_ok ? &lay_ws : nullptr,
                                ws_ok && ws_env == 1, &ch, s);
      if (rc != DVNR_OK) return rc;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = ch;
      have = true;
    }
    if (have) {
      if (ch.ws) p.lay = lay_ws;
      p.lay.ctas_per_sm = ch.ctas_per_sm;
      set_wave_tiles(p, ch.wave_tiles);
      interleaved = ch.interleaved && !p.sched;
    } else {
      if (ws_ok && ws_env == 1) p.lay = lay_ws;
      set_waves(p, m0, n);
      interleaved = interleave_env == 1 && !p.sched;
    }
  }
  const bool ws = p.lay.ws != 0;
  if (c->any_graph() && (c->wave_tiles != p.wave_tiles || c->ctas_per_sm != p.lay.ctas_per_sm ||
                  c->scheduled != (p.sched != nullptr) || c->interleaved != interleaved || c->ws != ws)) {
    DVNR_CUDA(cudaStreamSynchronize(s));
    c->drop_graph();
  }
  c->wave_tiles = p.wave_tiles;
  c->ctas_per_sm = p.lay.ctas_per_sm;
  c->scheduled = p.sched != nullptr;
  c->interleaved = interleaved;
  c->ws = ws;
  const int W = m0->mlp.width, F = m0->lv.F;
  DVNR_WF_DISPATCH(W, F, set_smem_attr, true, lay.smem_bytes);
  auto one_step = [&](cudaStream_t st) -> dvnr_status {
    if (interleaved) return launch_interleaved_step(p, W, F, n, c->d_adam, m0->n_store, h, st);
    dvnr_status rc = launch_train(p, W, F, n, st);
    if (rc != DVNR_OK) return rc;
    return launch_adam(c->d_adam, n, m0->n_store, h, st);
  };
  const int64_t step_launches = interleaved ? interleaved_launches(p, n) : (p.sched ? 3 : 2);
  int64_t left = steps;
  if (interleaved && left > 0) {
    // the call's first step has no pending update: it only trains, and the
    // interleaved steps that follow apply each update before the next
    // training of the model; the last update comes after them
    dvnr_status rc = launch_train(p, W, F, n, s);
    if (rc != DVNR_OK) return rc;
    count_eager_steps(1);
    left -= 1;
    rc = mp_train_steps(c, p, n, left, one_step, step_launches, s);
    if (rc != DVNR_OK) return rc;
    return launch_adam(c->d_adam, n, m0->n_store, h, s);
  }
  return mp_train_steps(c, p, n, left, one_step, step_launches, s);
}

dvnr_status mp_train_grad(dvnr_model m, const float* vol, const dvnr_train_cfg* cfg, uint32_t iter,
                          float S, const MpStepDebug& dbg, cudaStream_t s) {
  MpLayout lay;
  if (!make_layout(m, true, lay)) {
    set_error("FP16 path: configuration exceeds shared or tensor memory");
    return DVNR_E_UNSUPPORTED;
  }
  MpLayout lay_ws;
  if (train_ws_env() == 1 && make_layout_ws(m, lay_ws)) lay = lay_ws;
  MpModel hm{m->theta16, m->grad, vol, (int32_t)m->dims[0], (int32_t)m->dims[1], (int32_t)m->dims[2],
             0u, m->st};
  MpModel* d = nullptr;
  DVNR_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d), sizeof(MpModel), s));
  if (const cudaError_t e = cudaMemcpyAsync(d, &hm, sizeof(MpModel), cudaMemcpyHostToDevice, s); e != cudaSuccess) {
    dev_free_async(d, s);
    return cuda_status(e, "model descriptor");
  }
  MpParams p = base_params(m, lay, cfg);
  p.total_tiles = p.tiles_per_model;
  p.n_models = 1;
  p.sched = nullptr;
  p.models = d;
  p.explicit_iter = 1;
  p.iter = iter;
  p.loss_scale_override = S;
  p.dbg_y = dbg.y;
  p.dbg_dx0 = dbg.dx0;
  p.dbg_tgt = dbg.target;
  p.dbg_coords = dbg.coords;
  if (!(dbg.y && dbg.target && dbg.coords)) {
    p.dbg_y = nullptr;  // the per-sample outputs are written together
  }
  set_waves(p, m, 1);
  const int W = m->mlp.width, F = m->lv.F;
  DVNR_WF_DISPATCH(W, F, set_smem_attr, true, lay.smem_bytes);
  dvnr_status rc = launch_train(p, W, F, 1, s);
  dev_free_async(d, s);
  DVNR_CUDA(cudaStreamSynchronize(s));  // the host descriptor is released on return
  return rc;
}

dvnr_status mp_decode_rays(dvnr_model m, const RayFrame& rf, const RayBlock& rb, int64_t r0, int64_t nr,
                           float* out, cudaStream_t s) {
  return mp_decode_impl(m, nullptr, nr * rb.nk, 2, &rf, &rb, r0, nr, out, s);
}

dvnr_status mp_decode(dvnr_model m, const float* xyz, int64_t n, int grid_mode, float* out,
                      cudaStream_t s) {
  return mp_decode_impl(m, xyz, n, grid_mode, nullptr, nullptr, 0, 0, out, s);
}

dvnr_status mp_forward(dvnr_model m, const uint32_t* coords, int64_t n, float* y, cudaStream_t s) {
  return mp_decode_impl(m, nullptr, n, 3, nullptr, nullptr, 0, 0, y, s, coords);
}

dvnr_status mp_backward(dvnr_model m, const uint32_t* coords, const float* dy, int64_t n,
                        const float* scale_dev, float* dx0, cudaStream_t s) {
  MpLayout lay;
  if (!make_layout(m, true, lay)) {
    set_error("FP16 path: configuration exceeds shared or tensor memory");
    return DVNR_E_UNSUPPORTED;
  }
  MpLayout lay_ws;
  if (train_ws_env() == 1 && make_layout_ws(m, lay_ws)) lay = lay_ws;
  MpModel hm{m->theta16, m->grad, nullptr, (int32_t)m->dims[0], (int32_t)m->dims[1], (int32_t)m->dims[2],
             0u, m->st};
  MpModel* d = nullptr;
  DVNR_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d), sizeof(MpModel), s));
  if (const cudaError_t e = cudaMemcpyAsync(d, &hm, sizeof(MpModel), cudaMemcpyHostToDevice, s); e != cudaSuccess) {
    dev_free_async(d, s);
    return cuda_status(e, "model descriptor");
  }
  dvnr_train_cfg cfg{};
  cfg.batch = (int32_t)n;
  cfg.loss = DVNR_LOSS_L2;
  MpParams p = base_params(m, lay, &cfg);
  p.total_tiles = p.tiles_per_model;
  p.n_models = 1;
  p.sched = nullptr;
  p.models = d;
  p.explicit_iter = 1;
  p.ext_coords = coords;
  p.ext_dy = dy;
  p.ext_scale = scale_dev;
  p.dbg_dx0 = dx0;
  set_waves(p, m, 1);
  const int W = m->mlp.width, F = m->lv.F;
  DVNR_WF_DISPATCH(W, F, set_smem_attr, true, lay.smem_bytes);
  dvnr_status rc = launch_train(p, W, F, 1, s);
  dev_free_async(d, s);
  DVNR_CUDA(cudaStreamSynchronize(s));  // the host descriptor is released on return
  return rc;
}

dvnr_status mp_decode_impl(dvnr_model m, const float* xyz, int64_t n, int grid_mode, const RayFrame* rf,
                           const RayBlock* rb, int64_t r0, int64_t nr, float* out, cudaStream_t s,
                           const uint32_t* coords) {
  if (n <= 0) return DVNR_OK;
  MpLayout lay;
  if (!make_layout(m, false, lay)) {
    set_error("FP16 path: configuration exceeds shared or tensor memory");
    return DVNR_E_UNSUPPORTED;
  }
  MpDecodeParams p{};
  p.lv = m->lv;
  p.D = m->lv.in_dim;
  p.H = m->mlp.n_hidden;
  for (int k = 0; k <= m->mlp.n_hidden; ++k) p.w_off[k] = m->w_off[k];
  p.lay = lay;
  p.theta16 = m->theta16;
  p.st = m->st;
  p.n = n;
  p.n_tiles = (n + kTile - 1) / kTile;
  p.xyz = xyz;
  p.coords = coords;
  p.grid_mode = grid_mode;
  for (int a = 0; a < 3; ++a) {
    p.e[a] = m->box.hi[a] - m->box.lo[a];
    p.nstore[a] = m->dims[a];
    p.origin[a] = (float)(m->box.lo[a] - m->box.ghost);
  }
  p.ghost = m->box.ghost;
  p.out = out;
  p.first_wait_cycles = g_first_wait.load();
  p.div_e0 = make_fastdiv((uint64_t)p.e[0]);
  p.div_e1 = make_fastdiv((uint64_t)p.e[1]);
  for (int a = 0; a < 3; ++a) p.div_fix[a] = make_fastdiv(2 * (uint64_t)std::max<int64_t>(p.nstore[a] - 1, 1));
  if (rf) {
    p.rf = *rf;
    p.rb = *rb;
    p.r0 = r0;
    p.nr = nr;
    p.div_nr = make_fastdiv((uint64_t)nr);
    p.div_npx = make_fastdiv((uint64_t)rb->npx);
  }
  const int W = m->mlp.width, F = m->lv.F;
  DVNR_WF_DISPATCH(W, F, set_smem_attr, false, lay.smem_bytes);
  {
    ProfScope ps("decode_fp16", s);
    DVNR_WF_DISPATCH(W, F, launch_decode_wf, p, s);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

}  // namespace dvnr

extern "C" dvnr_status dvnr_debug_first_wait(int64_t cycles, int64_t* previous) {
  using namespace dvnr;
  if (cycles < -1) {
    set_error("cycles must be >= 0, or -1 for the default");
    return DVNR_E_INVALID;
  }
  const long long prev = g_first_wait.exchange(cycles == -1 ? kWaitCycles : (long long)cycles);
  if (previous) *previous = prev;
  return DVNR_OK;
}

extern "C" dvnr_status dvnr_selftest_umma(int32_t* mismatches_host) {
  using namespace dvnr;
  if (!mismatches_host) {
    set_error("NULL argument");
    return DVNR_E_INVALID;
  }
  int32_t* d = nullptr;
  DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&d), 5 * sizeof(int32_t)));
  cudaError_t e = cudaMemset(d, 0, 5 * sizeof(int32_t));
  if (e == cudaSuccess) {
    ProfScope ps("umma_selftest", 0);
    k_umma_selftest<<<1, 128>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(mismatches_host, d, 5 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  dev_free(d);
  if (e != cudaSuccess) return cuda_status(e, "dvnr_selftest_umma");
  return mismatches_host[4] ? DVNR_E_TIMEOUT : DVNR_OK;
}
