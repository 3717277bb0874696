// dvnr_internal.cuh -- shared declarations of the libdvnr translation units.
//
// Device helpers for the DVNR hot path (arXiv 2304.10516): counter-based
// sampling, 24-bit fixed-point lattice positions, the hash-grid corner index
// (Sec. 3, after Mueller et al. 2022), the model's device state, and the
// kernel launchers implemented in the other .cu files.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstring>
#include <string>

#include "../../include/dvnr.h"

namespace dvnr {

constexpr int kMaxLevels = 32;
constexpr int kMaxHidden = 8;
constexpr int kQTab = 4096;          // segments of the half-normal quantile table
constexpr uint32_t kFixOne = 1u << 24;  // unit coordinate u = m / 2^24
constexpr uint32_t kPurposeInit = 0x494E4954u;    // 'INIT'
constexpr uint32_t kPurposeSample = 0x53414D00u;  // 'SAM\0' + redraw attempt

// ---------------------------------------------------------------- errors ----
void set_error(const char* fmt, ...);
dvnr_status cuda_status(cudaError_t e, const char* what);
#define DVNR_CUDA(call)                                           \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return ::dvnr::cuda_status(e_, #call); \
  } while (0)

// ------------------------------------------------------------- profiling ----
// RAII bracket of one kernel launch: counts it and, while profiling is on,
// records CUDA events around it on its stream.
struct ProfScope {
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
bool profiling_on();
void count_launches(int64_t n);
// Device allocations of the library (alloc.cu): counted, and made to fail on
// request for tests of the cleanup paths. Freeing nullptr does nothing.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t dev_free_async(void* p, cudaStream_t s);
// dvnr_graph_stats counters of the grouped training's step graphs
void count_graph_capture();
void count_graph_replay();
void count_eager_steps(int64_t n);
void count_train_launch(bool ws);
// An NVTX range named after a public call, open for the call's duration (a
// host-side marker for profilers; without an attached tool it costs a
// branch).
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};
// Launches recorded into a CUDA graph are counted when the graph is replayed.
void set_capturing(bool on);
// A pinned host word, mapped into the device, that kernels add launch counts
// to (included in dvnr_launch_count once the device has written it); freed
// with its count kept. nullptr when pinned memory is not available.
unsigned long long* device_counter_new();
void device_counter_free(unsigned long long* p);

// ----------------------------------------------------------- level table ----
// Per-level layout of the hash-grid tables (kernel parameter, by value).
struct LevelTab {
  int32_t L, F, in_dim;
  uint32_t hash_mask;              // T - 1
  uint32_t dense_mask;             // bit l: level l stored densely
  uint32_t N[kMaxLevels];          // resolution N_l
  int64_t off[kMaxLevels];         // first parameter of level l
};

// Compact (ABI) parameter index -> index in the library's storage, where each
// level's table and the MLP block start on a 32-parameter boundary (so that a
// pair of adjacent FP16 entries is one aligned 8-byte load and a pair of FP32
// gradient entries one aligned 16-byte reduction). Block L is the MLP.
constexpr int64_t kParamAlign = 32;
struct LayoutMap {
  int32_t L;
  int64_t ext_off[kMaxLevels + 2];  // block starts in the compact layout; [L+1] = end
  int64_t int_off[kMaxLevels + 1];  // block starts in storage
};
__host__ __device__ inline int64_t ext_to_int(const LayoutMap& lm, int64_t i) {
  int l = 0;
  while (l < lm.L && i >= lm.ext_off[l + 1]) ++l;
  return lm.int_off[l] + (i - lm.ext_off[l]);
}

// ------------------------------------------------------- device state ------
// Per-model state that lives on the device so that whole training steps can
// be captured in a CUDA graph and replayed.
// Bits of ModelState::overflow: the step's gradient is unusable and Adam
// skips the step (and clears the gradient). A non-finite gradient also halves
// the FP16 loss scale; an aborted step (a bounded wait gave up) does not.
constexpr uint32_t kNonFiniteGrad = 1u;
constexpr uint32_t kStepAborted = 2u;

struct ModelState {
  uint32_t enc_min, enc_max;  // order-preserving encodings of the value range
  uint32_t nonfinite;         // training volume held NaN/Inf
  uint32_t overflow;          // kNonFiniteGrad | kStepAborted of this step
  float loss_scale;           // dynamic loss scale S (FP16 path)
  uint32_t good_steps;        // finite steps since the last scale change
  uint32_t iter;              // iterations drawn (Philox counter word 1)
  uint32_t adam_t;            // Adam steps applied
  uint32_t skipped;           // steps skipped for non-finite gradients
  uint32_t done_blocks;       // Adam last-block counter
  float loss_sum;             // sum of per-sample losses of this step
  float last_loss;            // mean loss of the last completed step
  uint32_t timeouts;          // bounded device waits that gave up
  // iteration budget and early stop of the current training call (Sec. 3.2)
  uint32_t stop_at;           // the call ends this model's training at iter == stop_at
  float loss_ema;             // moving average of the loss in this call (< 0: none yet)
  uint32_t stopped;           // the moving average fell below the stop threshold
  float ext_scale;            // loss scale of the last dvnr_backward (FP16 path)
};

// A model takes part in a training step while its call's budget lasts and it
// has not met the stop threshold. Every kernel of a step evaluates this on
// the same state: only the last block of Adam changes it, after all the
// step's other reads.
__host__ __device__ inline bool model_active(const ModelState* st) {
  return st->iter < st->stop_at && st->stopped == 0u;
}

__host__ __device__ inline uint32_t float_to_ordered(float f) {
#ifdef __CUDA_ARCH__
  uint32_t b = __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float ordered_to_float(uint32_t e) {
  uint32_t b = (e & 0x80000000u) ? (e & 0x7FFFFFFFu) : ~e;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

// ------------------------------------------------------------ the model ----
struct Fp32Workspace {
  int64_t batch = 0;
  float* x0 = nullptr;     // batch x in_dim
  float* act = nullptr;    // n_hidden x batch x width  (H_1 .. H_H)
  float* dz = nullptr;     // 2 x batch x width (ping-pong)
  float* dx0 = nullptr;    // batch x in_dim
  float* tgt = nullptr;    // batch
  uint32_t* coords = nullptr;  // batch x 3
  void* base = nullptr;
};

}  // namespace dvnr

struct dvnr_model_s {
  int device = 0;
  // process-wide unique id, never reused: caches keyed on models compare ids,
  // since a destroyed model's handle address can come back for a new model
  uint64_t uid = 0;
  dvnr_box box{};
  dvnr_enc_cfg enc{};
  dvnr_mlp_cfg mlp{};
  dvnr::LevelTab lv{};
  int64_t dims[3] = {0, 0, 0};  // stored voxels per axis (ghost included)
  int64_t n_enc = 0, n_mlp = 0, n_params = 0;  // compact (ABI) counts
  int64_t n_store = 0;          // parameters in storage (level tables padded)
  dvnr::LayoutMap lmap{};       // compact index -> storage index
  int64_t w_off[dvnr::kMaxHidden + 1] = {};
  double glorot[dvnr::kMaxHidden + 1] = {};  // init limit of each matrix
  // parameter block: theta | m1 | m2 | grad (fp32), theta16, state, qtab
  void* block = nullptr;
  size_t block_bytes = 0;       // device bytes of `block`
  float* theta = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  __half* theta16 = nullptr;
  dvnr::ModelState* st = nullptr;
  int32_t* qtab = nullptr;
  float qtab_sigma = -1.f;
  int32_t precision = DVNR_FP32;
  bool scale_initialized = false;  // FP16 loss scale set for this model
  // frozen: only the FP16 parameters and the state remain (theta, m1, m2,
  // grad and qtab are NULL); decodes and renders in FP16, cannot train
  bool frozen = false;
  dvnr::Fp32Workspace ws;
  void* mp = nullptr;              // FP16 path resources (mp_path.cu)
  float* grid_ws = nullptr;  // decoded grid for rendering
  size_t grid_ws_elems = 0;
};

namespace dvnr {

// ------------------------------------------------------- device helpers ----
#ifdef __CUDACC__
// Philox-4x32-10 (Salmon et al. 2011), ten rounds with bumped keys.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Lattice position of a fixed-point coordinate on n cells: p = m n / 2^24,
// base = min(floor(p), n - 1), frac = p - base (exact in float).
__device__ __forceinline__ void lattice(uint32_t m, uint32_t n, uint32_t& base, float& frac) {
  const uint64_t p = (uint64_t)m * n;
  uint32_t b = (uint32_t)(p >> 24);
  b = b < n - 1 ? b : n - 1;
  base = b;
  frac = (float)(uint32_t)(p - ((uint64_t)b << 24)) * (1.0f / 16777216.0f);
}

// Table index of vertex (x, y, z) of level l: dense x + y(N+1) + z(N+1)^2,
// hashed (x * 1 xor y * 2654435761 xor z * 805459861) mod T (Mueller et al.).
__device__ __forceinline__ uint32_t corner_index(const LevelTab& lv, int l, uint32_t x, uint32_t y,
                                                 uint32_t z) {
  if ((lv.dense_mask >> l) & 1u) {
    const uint32_t s = lv.N[l] + 1u;
    return x + s * (y + s * z);
  }
  return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & lv.hash_mask;
}

// The 8 corners of the cell with lower corner (x, y, z) at level l, corner k
// = (x + (k&1), y + ((k>>1)&1), z + ((k>>2)&1)): the values of corner_index,
// formed from one base per level (dense: base + {0, 1, s, s + 1, s^2, ...};
// hashed: the y and z products once each, (y + 1) P = y P + P mod 2^32).
__device__ __forceinline__ void corner_indices8(const LevelTab& lv, int l, uint32_t x, uint32_t y, uint32_t z,
                                                uint32_t (&idx)[8]) {
  if ((lv.dense_mask >> l) & 1u) {
    const uint32_t s = lv.N[l] + 1u, s2 = s * s;
    const uint32_t b = x + s * (y + s * z);
#pragma unroll
    for (int k = 0; k < 8; ++k) idx[k] = b + (uint32_t)(k & 1) + ((k >> 1) & 1 ? s : 0u) + ((k >> 2) & 1 ? s2 : 0u);
  } else {
    const uint32_t hy0 = y * 2654435761u, hy1 = hy0 + 2654435761u;
    const uint32_t hz0 = z * 805459861u, hz1 = hz0 + 805459861u;
    const uint32_t msk = lv.hash_mask;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      idx[k] = ((x + (uint32_t)(k & 1)) ^ ((k >> 1) & 1 ? hy1 : hy0) ^ ((k >> 2) & 1 ? hz1 : hz0)) & msk;
  }
}

// Sampling parameters of one model slot in one step (Sec. 3.2-3.3).
struct SampleParams {
  uint2 key;           // seed
  uint32_t model;      // model slot
  int32_t n_bnd;       // floor(lambda batch) boundary samples first
  const int32_t* qtab; // half-normal quantile table, kQTab + 1 knots
};

// Fixed-point coordinates of sample i of iteration `iter`.
__device__ __forceinline__ uint3 draw_sample(const SampleParams& sp, uint32_t i, uint32_t iter) {
  if ((int32_t)i >= sp.n_bnd) {
    const uint4 r = philox(make_uint4(i, iter, sp.model, kPurposeSample), sp.key);
    return make_uint3(r.x >> 8, r.y >> 8, r.z >> 8);
  }
  for (uint32_t attempt = 0;; ++attempt) {
    const uint4 r = philox(make_uint4(i, iter, sp.model, kPurposeSample + attempt), sp.key);
    const uint32_t face = __umulhi(r.x, 6u);
    const uint32_t axis = face >> 1, side = face & 1u;
    const uint32_t u24 = r.y >> 8, k = u24 >> 12, fr = u24 & 4095u;
    const int64_t q0 = __ldg(sp.qtab + k), q1 = __ldg(sp.qtab + k + 1);
    int64_t off = q0 + (((q1 - q0) * (int64_t)fr) >> 12);
    if (off > (int64_t)kFixOne && attempt < 255) continue;
    if (off > (int64_t)kFixOne) off = kFixOne;
    const uint32_t c = side ? kFixOne - (uint32_t)off : (uint32_t)off;
    const uint32_t a = r.z >> 8, b = r.w >> 8;
    if (axis == 0) return make_uint3(c, a, b);
    if (axis == 1) return make_uint3(a, c, b);
    return make_uint3(a, b, c);
  }
}

// Trilinear lookup of a stored block at a fixed-point coordinate: position
// u (n - 1) per axis (the block spans [0,1] between its outer voxel centres).
// vol_fetch issues the eight corner loads; vol_interp combines them, so the
// loads can stay in flight while other work runs.
struct VolCorners {
  float v[8];
  float fx, fy, fz;
};

__device__ __forceinline__ VolCorners vol_fetch(const float* __restrict__ vol, int nx, int ny, int nz,
                                                uint3 m) {
  VolCorners c;
  uint32_t bx, by, bz;
  lattice(m.x, (uint32_t)(nx - 1), bx, c.fx);
  lattice(m.y, (uint32_t)(ny - 1), by, c.fy);
  lattice(m.z, (uint32_t)(nz - 1), bz, c.fz);
  const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
  const float* p = vol + bz * sz + by * sy + bx;
  // evict-first: a training volume is read at eight random corners per sample
  // and is larger than the share of L2 the tables and gradients need
  c.v[0] = __ldcs(p);
  c.v[1] = __ldcs(p + 1);
  c.v[2] = __ldcs(p + sy);
  c.v[3] = __ldcs(p + sy + 1);
  c.v[4] = __ldcs(p + sz);
  c.v[5] = __ldcs(p + sz + 1);
  c.v[6] = __ldcs(p + sz + sy);
  c.v[7] = __ldcs(p + sz + sy + 1);
  return c;
}

__device__ __forceinline__ float vol_interp(const VolCorners& c) {
  const float gx = 1.f - c.fx, gy = 1.f - c.fy, gz = 1.f - c.fz;
  return gz * (gy * (gx * c.v[0] + c.fx * c.v[1]) + c.fy * (gx * c.v[2] + c.fx * c.v[3])) +
         c.fz * (gy * (gx * c.v[4] + c.fx * c.v[5]) + c.fy * (gx * c.v[6] + c.fx * c.v[7]));
}

__device__ __forceinline__ float volume_trilinear(const float* __restrict__ vol, int nx, int ny,
                                                  int nz, uint3 m) {
  return vol_interp(vol_fetch(vol, nx, ny, nz, m));
}

// Ray lattice of direct volume rendering (Sec. 4.3 reading): orthographic
// rays along +z through pixel centres over the frame [lo - 1/2, hi - 1/2),
// spr samples at the centres of spr equal steps in z. A block owns the
// pixels px0 .. px0+npx-1, py0 .. py0+npy-1 whose ray centre lies in its box
// and the samples k0 .. k0+nk-1 inside it; its rays are numbered row-major
// over that footprint. Positions use these single-precision expressions on
// the host and the device alike.
struct RayFrame {
  float lo[3], hi[3];
  int32_t w, h, spr;
};
struct RayBlock {
  float origin[3];  // global coordinate of the block's stored voxel 0 (lo - ghost)
  int32_t nstore[3];
  int32_t px0, npx, py0, npy, k0, nk;
};
__host__ __device__ __forceinline__ float frame_x(const RayFrame& f, int px) {
  return (f.lo[0] - 0.5f) + ((px + 0.5f) * (f.hi[0] - f.lo[0])) / (float)f.w;
}
__host__ __device__ __forceinline__ float frame_y(const RayFrame& f, int py) {
  return (f.lo[1] - 0.5f) + ((py + 0.5f) * (f.hi[1] - f.lo[1])) / (float)f.h;
}
__host__ __device__ __forceinline__ float frame_z(const RayFrame& f, int k) {
  return (f.lo[2] - 0.5f) + ((k + 0.5f) * (f.hi[2] - f.lo[2])) / (float)f.spr;
}

// Division of unsigned 64-bit integers by a divisor d >= 1 fixed for a
// launch, by a multiply-high with the reciprocal m = floor((2^64 - 1) / d)
// and a remainder correction (division by invariant integers, Granlund and
// Montgomery 1994): num * m / 2^64 is below num / d by less than 2, so the
// quotient estimate is q, q - 1 or q - 2 and at most two corrections make it
// exact for every num < 2^64.
struct FastDiv {
  uint64_t d, m;
};
inline FastDiv make_fastdiv(uint64_t d) {
  if (d == 0) d = 1;
  return FastDiv{d, ~0ull / d};
}
__device__ __forceinline__ uint64_t fdiv(uint64_t num, const FastDiv& f) {
  uint64_t q = __umul64hi(num, f.m);
  uint64_t r = num - q * f.d;
  if (r >= f.d) {
    ++q;
    r -= f.d;
  }
  if (r >= f.d) ++q;
  return q;
}

__device__ __forceinline__ void value_range(const ModelState* st, float& vmin, float& inv_range) {
  vmin = ordered_to_float(st->enc_min);
  const float vmax = ordered_to_float(st->enc_max);
  inv_range = vmax > vmin ? 1.0f / (vmax - vmin) : 0.0f;
}
#endif  // __CUDACC__

// -------------------------------------------------------------- launchers ---
// Model-independent kernels (util.cu)
dvnr_status launch_init_params(dvnr_model m, uint64_t seed, cudaStream_t s);
dvnr_status launch_refresh_half(dvnr_model m, cudaStream_t s);
dvnr_status launch_widen_half(dvnr_model m, cudaStream_t s);
dvnr_status launch_begin_call(ModelState* st, uint32_t budget, cudaStream_t s);
// Load a caller-given gradient (compact layout, unscaled) into the model's
// gradient buffer as Adam expects it: times the loss scale on the FP16 path,
// a non-finite value flagged as kNonFiniteGrad.
dvnr_status launch_load_grad(dvnr_model m, const float* grad_in, bool mixed, cudaStream_t s);
// Look up the device address of dvnr_error_stats_noalloc's scratch array on
// the current device now (once per device).
dvnr_status prime_err_scratch();
dvnr_status launch_minmax(const float* vol, int64_t n, ModelState* st, cudaStream_t s);
dvnr_status launch_error_stats(const float* a, const float* b, int64_t n, double* out_dev,
                               cudaStream_t s);
dvnr_status launch_corner_indices(dvnr_model m, const uint32_t* coords, int64_t n, uint32_t* idx,
                                  cudaStream_t s);

struct AdamModelPtrs {
  float* theta;
  float* m1;
  float* m2;
  float* grad;
  __half* theta16;
  ModelState* st;
};
struct AdamHyper {
  float lr, beta1, beta2, eps, weight_decay;
  float inv_batch;
  int32_t mixed, growth_interval;
  int32_t gated;               // skip models that are not model_active
  float stop_loss, stop_decay; // early stop (stop_loss 0: off)
  // the gradient came from the caller (dvnr_adam_step): no samples were
  // drawn and no loss was taken, so the iteration count, the last loss and
  // its moving average stay as they are
  int32_t external;
  // launch-shape trials: the memory traffic of a step (read g, theta, m, v;
  // write theta, m, v, the FP16 copy, a cleared g) with every value written
  // back unchanged (the gradient cleared) and no counter touched
  int32_t dry;
};
dvnr_status launch_adam(const AdamModelPtrs* models_dev, int n_models, int64_t n_params,
                        const AdamHyper& h, cudaStream_t s);

// Plain FP32 path (fp32_path.cu)
struct Fp32StepArgs {
  dvnr_model m;
  const float* vol;
  SampleParams sp;
  int32_t batch;
  int32_t loss;
  bool explicit_iter;
  uint32_t iter;
  bool gated;  // every kernel of the step returns at once when !model_active
  // optional debug outputs
  float* y_out;
  float* dx0_out;
  float* tgt_out;
  uint32_t* coords_out;
  // backward at caller-given points (dvnr_backward): fixed-point coordinates
  // (batch x 3) instead of drawn samples and the upstream dL/dy (batch)
  // instead of the loss; no volume. nullptr in training.
  const uint32_t* ext_coords = nullptr;
  const float* ext_dy = nullptr;
};
dvnr_status fp32_ensure_workspace(dvnr_model m, int64_t batch);
dvnr_status fp32_forward_backward(const Fp32StepArgs& a, cudaStream_t s);
// raw: write the network output y itself instead of y (vmax - vmin) + vmin
dvnr_status fp32_decode_unit(dvnr_model m, const uint32_t* coords, const float* xyz, int64_t n,
                             int grid_mode, float* out, cudaStream_t s, bool raw = false);

// Render (render.cu)
struct RenderBlock {
  float lo[3], hi[3];  // owned box, global voxel indices
  int32_t e[3];        // owned voxels per axis
  int32_t pad;
  const float* grid;   // decoded owned grid, x fastest
};
dvnr_status launch_render(const RenderBlock* blocks_dev, int n_blocks, const float lo[3],
                          const float hi[3], const dvnr_tf& tf, int w, int h, int spr,
                          float* rgba, cudaStream_t s);
// Same encoding and MLP configuration (api.cu).
bool same_arch(const dvnr_model a, const dvnr_model b);

// Direct INR ray-marching (render_inr.cu): same camera and transfer function
// as launch_render, values from the models' networks at the ray samples.
// All models share one precision; FP16 models also one architecture.
dvnr_status render_inr(const dvnr_model* models, int n, const float* frame_lo, const float* frame_hi,
                       const dvnr_tf& tf, int w, int h, int spr, float* rgba, cudaStream_t s);
// Sort-last blend (render_inr.cu): images rgba[order[0]] (front) ..
// rgba[order[n-1]] (back), npix float4 pixels each, into out; synchronises.
dvnr_status composite(const float* const* rgba, const int* order, int n, int64_t npix, float* out,
                      cudaStream_t s);
dvnr_status launch_state_reset(ModelState* st, float loss_scale, cudaStream_t s);
dvnr_status launch_state_reset_scale(ModelState* st, float loss_scale, cudaStream_t s);
// S for a backward at given points: loss_scale > 0 is taken as it is, else
// 2^round(-log2 max|dy|) (1 when dy is all zero or not finite), so that the
// largest scaled output gradient is about 1 as in training; stored in
// m->st->ext_scale.
dvnr_status launch_ext_scale(dvnr_model m, const float* dy, int64_t n, float loss_scale, cudaStream_t s);
// Master weights from a device array in the compact layout, FP16 copy refreshed.
dvnr_status launch_load_params(dvnr_model m, const float* params, cudaStream_t s);
// As launch_finish_grad with the loss scale read from *scale_dev.
dvnr_status launch_finish_grad_dev(dvnr_model m, const float* scale_dev, float* grad_out, cudaStream_t s);
dvnr_status launch_finish_grad(dvnr_model m, float loss_scale_used, float inv_batch, float* grad_out,
                               float* loss_out, cudaStream_t s);

}  // namespace dvnr
