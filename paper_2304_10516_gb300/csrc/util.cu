// util.cu -- initialisation, value-range pre-pass, fused Adam, FP64 error
// reduction and the corner-index probe of libdvnr.
#include <cstring>
#include <mutex>

#include "dvnr_internal.cuh"

namespace dvnr {

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// Parameter initialisation (the paper is silent; Mueller et al. tables
// U(-1e-4, 1e-4), Glorot-uniform MLP). u = (r0 >> 8) 2^-24 from Philox block
// {i_lo, i_hi, 0, 'INIT'} keyed by the seed; v = lo + (hi - lo) u computed in
// FP64 with explicit round-to-nearest operations, then rounded to binary32.
struct InitArgs {
  float* theta;
  __half* theta16;
  int64_t n_params, n_enc;
  int64_t bound[kMaxHidden + 1];  // end (exclusive, compact index) of matrix k
  double limit[kMaxHidden + 1];
  int32_t n_mats;
  uint2 key;
  LayoutMap lmap;
};

__global__ void k_init_params(InitArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_params;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox(make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, kPurposeInit),
                           a.key);
    const double u = (double)(r.x >> 8) * (1.0 / 16777216.0);
    double lo, hi;
    if (i < a.n_enc) {
      lo = -1e-4;
      hi = 1e-4;
    } else {
      int k = 0;
      while (k < a.n_mats - 1 && i >= a.bound[k]) ++k;
      lo = -a.limit[k];
      hi = a.limit[k];
    }
    const double span = __dsub_rn(hi, lo);
    const double v = __dadd_rn(lo, __dmul_rn(span, u));
    const float f = __double2float_rn(v);
    const int64_t j = ext_to_int(a.lmap, i);
    a.theta[j] = f;
    a.theta16[j] = __float2half_rn(f);
  }
}

__global__ void k_refresh_half(const float* __restrict__ theta, __half* __restrict__ theta16,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    theta16[i] = __float2half_rn(theta[i]);
}

__global__ void k_widen_half(const __half* __restrict__ theta16, float* __restrict__ theta, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    theta[i] = __half2float(theta16[i]);
}

// Value range of a training volume (Sec. 3.1 normalises values by the
// partition's min and max, ghost layer included) and a NaN/Inf check.
__global__ void k_minmax(const float* __restrict__ v, int64_t n, ModelState* st) {
  float lo = INFINITY, hi = -INFINITY;
  uint32_t bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = __ldg(v + i);
    if (!isfinite(x)) {
      bad = 1;
      continue;
    }
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (lo <= hi) {
      atomicMin(&st->enc_min, float_to_ordered(lo));
      atomicMax(&st->enc_max, float_to_ordered(hi));
    }
    if (bad) atomicOr(&st->nonfinite, 1u);
  }
}

// FP64 reduction of sum (a-b)^2 and max |a-b| (Sec. 5: PSNR from the MSE).
__global__ void k_error_stats(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                              double* out) {
  double s = 0.0, mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)__ldg(a + i) - (double)__ldg(b + i);
    s += d * d;
    mx = fmax(mx, fabs(d));
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double ss[kThreads / 32], sm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, m = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t += ss[w];
      m = fmax(m, sm[w]);
    }
    atomicAdd(out, t);
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(out + 1),
              (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_corner_indices(LevelTab lv, const uint32_t* __restrict__ coords, int64_t n,
                                 uint32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t mx = coords[3 * i], my = coords[3 * i + 1], mz = coords[3 * i + 2];
    for (int l = 0; l < lv.L; ++l) {
      uint32_t bx, by, bz;
      float f;
      lattice(mx, lv.N[l], bx, f);
      lattice(my, lv.N[l], by, f);
      lattice(mz, lv.N[l], bz, f);
      for (int k = 0; k < 8; ++k)
        idx[(i * lv.L + l) * 8 + k] =
            corner_index(lv, l, bx + (k & 1), by + ((k >> 1) & 1), bz + ((k >> 2) & 1));
    }
  }
}

// Fused Adam over every parameter of every model of a step (Sec. 3.6:
// beta1, beta2, eps, L2 weight decay added to the gradient; Kingma & Ba bias
// correction). One HBM pass: read grad, theta, m, v; write theta, m, v, the
// FP16 copy and a zeroed grad. A step whose gradient held a non-finite value
// (flag set by the training kernels) is skipped and, on the FP16 path, halves
// the loss scale; growth_interval finite steps double it. The last block of
// each model updates the model's step counters.
__global__ void __launch_bounds__(kThreads) k_adam(const AdamModelPtrs* __restrict__ models,
                                                   int64_t n, AdamHyper h) {
  const AdamModelPtrs md = models[blockIdx.y];
  ModelState* st = md.st;
  if (h.gated && !model_active(st)) return;  // budget spent or stopped: no work, no counters
  const uint32_t ov = *((volatile uint32_t*)&st->overflow);
  const bool skip = ov != 0u && !h.dry;
  const float S = h.mixed ? st->loss_scale : 1.0f;
  const float inv_S = 1.0f / S;
  const uint32_t t = st->adam_t + 1u;
  // bias corrections 1 - beta^t. Formed as 1 - powf(beta, t) they cancel:
  // one rounding of beta2^t near 1 is up to ~1.5e-5 of 1 - beta2^t in the
  // first steps (beta2 = 0.999). With beta = 1 - d (d exact for beta >= 1/2)
  // 1 - beta^t = -expm1(t log1p(-d)), which keeps a few ulps.
  const float bc1 = -expm1f((float)t * log1pf(-(1.0f - h.beta1)));
  const float bc2 = -expm1f((float)t * log1pf(-(1.0f - h.beta2)));
  const float ib1 = 1.0f - h.beta1, ib2 = 1.0f - h.beta2;
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float4* g4 = reinterpret_cast<float4*>(md.grad);
  if (!skip) {
    float4* th4 = reinterpret_cast<float4*>(md.theta);
    float4* m14 = reinterpret_cast<float4*>(md.m1);
    float4* m24 = reinterpret_cast<float4*>(md.m2);
    for (int64_t i = tid; i < n4; i += stride) {
      // streaming loads/stores (evict-first): this pass touches every optimiser
      // word once per step and would otherwise push the tables, the FP16 copy
      // and the gradients that the next step gathers out of L2
      float4 g = __ldcs(g4 + i), th = __ldcs(th4 + i), a = __ldcs(m14 + i), b = __ldcs(m24 + i);
      float* gp = &g.x;
      float* tp = &th.x;
      float* ap = &a.x;
      float* bp = &b.x;
      if (!h.dry) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float gg = gp[j] * inv_S + h.weight_decay * tp[j];
          ap[j] = h.beta1 * ap[j] + ib1 * gg;
          bp[j] = h.beta2 * bp[j] + ib2 * gg * gg;
          tp[j] -= h.lr * (ap[j] / bc1) / (sqrtf(bp[j] / bc2) + h.eps);
        }
      }
      __stcs(th4 + i, th);
      __stcs(m14 + i, a);
      __stcs(m24 + i, b);
      g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      __half2* h2 = reinterpret_cast<__half2*>(md.theta16) + 2 * i;
      h2[0] = __floats2half2_rn(th.x, th.y);
      h2[1] = __floats2half2_rn(th.z, th.w);
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) {
      const float gg = md.grad[i] * inv_S + h.weight_decay * md.theta[i];
      const float a = h.dry ? md.m1[i] : h.beta1 * md.m1[i] + ib1 * gg;
      const float b = h.dry ? md.m2[i] : h.beta2 * md.m2[i] + ib2 * gg * gg;
      const float th = h.dry ? md.theta[i] : md.theta[i] - h.lr * (a / bc1) / (sqrtf(b / bc2) + h.eps);
      md.m1[i] = a;
      md.m2[i] = b;
      md.theta[i] = th;
      md.theta16[i] = __float2half_rn(th);
      md.grad[i] = 0.f;
    }
  } else {
    for (int64_t i = tid; i < n4; i += stride) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) md.grad[i] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !h.dry) {
    __threadfence();
    const uint32_t done = atomicAdd(&st->done_blocks, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      if (skip) {
        st->skipped += 1u;
        st->good_steps = 0u;
        if (h.mixed && (ov & kNonFiniteGrad)) st->loss_scale = S * 0.5f;
      } else {
        st->adam_t = t;
        if (h.mixed) {
          const uint32_t gs = st->good_steps + 1u;
          if ((int32_t)gs >= h.growth_interval) {
            st->loss_scale = S * 2.0f;
            st->good_steps = 0u;
          } else {
            st->good_steps = gs;
          }
        }
      }
      const float L = st->loss_sum * h.inv_batch;
      if (!h.external) st->last_loss = L;
      if (!skip && !h.external) {
        // moving average of the loss over the finite steps of the call and
        // the early-stop test (Sec. 3.2)
        const float e = st->loss_ema < 0.f ? L : __fadd_rn(__fmul_rn(h.stop_decay, st->loss_ema),
                                                           __fmul_rn(1.0f - h.stop_decay, L));
        st->loss_ema = e;
        if (h.stop_loss > 0.f && e < h.stop_loss) st->stopped = 1u;
      }
      st->loss_sum = 0.f;
      st->overflow = 0u;
      if (!h.external) st->iter += 1u;
      st->done_blocks = 0u;
    }
  }
}

// Reset the optimiser counters of a model, keeping its value range.
__global__ void k_state_reset(ModelState* st, float loss_scale) {
  st->nonfinite = 0u;
  st->overflow = 0u;
  st->loss_scale = loss_scale;
  st->good_steps = 0u;
  st->iter = 0u;
  st->adam_t = 0u;
  st->skipped = 0u;
  st->done_blocks = 0u;
  st->loss_sum = 0.f;
  st->last_loss = 0.f;
  st->timeouts = 0u;
  st->stop_at = 0xFFFFFFFFu;
  st->loss_ema = -1.f;
  st->stopped = 0u;
}

// Start of a training call: the budget runs from the current iteration (the
// end saturates at 2^32 - 1), the moving average starts afresh and the
// timeout count starts at zero (it reports this call's bounded waits).
__global__ void k_begin_call(ModelState* st, uint32_t budget) {
  const uint32_t it = st->iter;
  st->stop_at = budget > 0xFFFFFFFFu - it ? 0xFFFFFFFFu : it + budget;
  st->loss_ema = -1.f;
  st->stopped = 0u;
  st->timeouts = 0u;
}

// Hand out the gradient of one forward/backward without an optimiser step:
// grad_out = grad / S, loss_out = loss_sum / B; then clear the accumulators.
__global__ void k_finish_grad(float* __restrict__ grad, int64_t n_params,
                              LayoutMap lmap, float inv_S, float* __restrict__ grad_out,
                              ModelState* st, float inv_batch, float* __restrict__ loss_out,
                              const float* __restrict__ scale_dev) {
  if (scale_dev) inv_S = 1.0f / *scale_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // each storage entry belongs to one compact index, read and cleared by the
  // same thread; the padding between level tables is never written
  for (int64_t i = t0; i < n_params; i += stride) {
    const int64_t j = ext_to_int(lmap, i);
    if (grad_out) grad_out[i] = grad[j] * inv_S;
    grad[j] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t done = atomicAdd(&st->done_blocks, 1u);
    if (done == gridDim.x - 1) {
      if (loss_out) *loss_out = st->loss_sum * inv_batch;
      st->loss_sum = 0.f;
      st->overflow = 0u;
      st->done_blocks = 0u;
    }
  }
}

// grad[storage j] = g_in[compact i] S (S the loss scale on the FP16 path, else
// 1); a value that is or becomes non-finite flags the step. Storage padding is
// never written (it stays zero).
__global__ void k_load_grad(float* __restrict__ grad, const float* __restrict__ g_in, int64_t n_params,
                            LayoutMap lmap, ModelState* st, int mixed) {
  const float S = mixed ? st->loss_scale : 1.0f;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_params;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = g_in[i] * S;
    bad |= !isfinite(g);
    grad[ext_to_int(lmap, i)] = g;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->overflow, kNonFiniteGrad);
}

// Loss scale of a backward at given points: one block, max |dy| over n.
__global__ void __launch_bounds__(kThreads) k_ext_scale(const float* __restrict__ dy, int64_t n,
                                                        ModelState* st) {
  float mx = 0.f;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = fabsf(dy[i]);
    bad |= !isfinite(v);
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float sm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, sm[w]);
    float S = 1.0f;
    if (!bad && mx > 0.f) {
      int e = 0;
      frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1): 2^(1-e) puts the largest scaled value in [1, 2)
      e = 1 - e;
      e = e < -24 ? -24 : (e > 40 ? 40 : e);
      S = ldexpf(1.0f, e);
    }
    st->ext_scale = S;
  }
}

__global__ void k_set_ext_scale(ModelState* st, float S) { st->ext_scale = S; }

// theta[storage j] = params[compact i] and its binary16 copy.
__global__ void k_load_params(float* __restrict__ theta, __half* __restrict__ theta16,
                              const float* __restrict__ params, int64_t n_params, LayoutMap lmap) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_params;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = ext_to_int(lmap, i);
    const float v = params[i];
    theta[j] = v;
    theta16[j] = __float2half_rn(v);
  }
}

__global__ void k_state_set_scale(ModelState* st, float loss_scale) {
  st->loss_scale = loss_scale;
  st->good_steps = 0u;
}

}  // namespace

dvnr_status launch_state_reset_scale(ModelState* st, float loss_scale, cudaStream_t s) {
  {
    ProfScope ps_("state_reset", s);
    k_state_set_scale<<<1, 1, 0, s>>>(st, loss_scale);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_state_reset(ModelState* st, float loss_scale, cudaStream_t s) {
  {
    ProfScope ps_("state_reset", s);
    k_state_reset<<<1, 1, 0, s>>>(st, loss_scale);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_finish_grad(dvnr_model m, float loss_scale_used, float inv_batch, float* grad_out,
                               float* loss_out, cudaStream_t s) {
  {
    ProfScope ps_("finish_grad", s);
    k_finish_grad<<<grid_for(m->n_store, kThreads), kThreads, 0, s>>>(
      m->grad, m->n_params, m->lmap, 1.0f / loss_scale_used, grad_out, m->st,
      inv_batch, loss_out, nullptr);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_load_grad(dvnr_model m, const float* grad_in, bool mixed, cudaStream_t s) {
  {
    ProfScope ps_("load_grad", s);
    k_load_grad<<<grid_for(m->n_params, kThreads), kThreads, 0, s>>>(m->grad, grad_in, m->n_params, m->lmap,
                                                                     m->st, mixed ? 1 : 0);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_ext_scale(dvnr_model m, const float* dy, int64_t n, float loss_scale, cudaStream_t s) {
  {
    ProfScope ps_("ext_scale", s);
    if (loss_scale > 0.f)
      k_set_ext_scale<<<1, 1, 0, s>>>(m->st, loss_scale);
    else
      k_ext_scale<<<1, kThreads, 0, s>>>(dy, n, m->st);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_load_params(dvnr_model m, const float* params, cudaStream_t s) {
  {
    ProfScope ps_("load_params", s);
    k_load_params<<<grid_for(m->n_params, kThreads), kThreads, 0, s>>>(m->theta, m->theta16, params,
                                                                       m->n_params, m->lmap);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_finish_grad_dev(dvnr_model m, const float* scale_dev, float* grad_out, cudaStream_t s) {
  {
    ProfScope ps_("finish_grad", s);
    k_finish_grad<<<grid_for(m->n_store, kThreads), kThreads, 0, s>>>(
      m->grad, m->n_params, m->lmap, 1.0f, grad_out, m->st, 0.f, nullptr, scale_dev);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_init_params(dvnr_model m, uint64_t seed, cudaStream_t s) {
  InitArgs a;
  a.theta = m->theta;
  a.theta16 = m->theta16;
  a.n_params = m->n_params;
  a.n_enc = m->n_enc;
  a.n_mats = m->mlp.n_hidden + 1;
  a.lmap = m->lmap;
  // matrix bounds in compact indices: storage offset minus the MLP block shift
  const int64_t shift = m->lmap.int_off[m->lmap.L] - m->lmap.ext_off[m->lmap.L];
  for (int k = 0; k <= m->mlp.n_hidden; ++k) {
    a.bound[k] = (k < m->mlp.n_hidden) ? m->w_off[k + 1] - shift : m->n_params;
    a.limit[k] = m->glorot[k];
  }
  a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  {
    ProfScope ps_("init_params", s);
    k_init_params<<<grid_for(m->n_params, kThreads), kThreads, 0, s>>>(a);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_refresh_half(dvnr_model m, cudaStream_t s) {
  {
    ProfScope ps_("refresh_half", s);
    k_refresh_half<<<grid_for(m->n_store, kThreads), kThreads, 0, s>>>(m->theta, m->theta16,
                                                                    m->n_store);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_widen_half(dvnr_model m, cudaStream_t s) {
  {
    ProfScope ps_("widen_half", s);
    k_widen_half<<<grid_for(m->n_store, kThreads), kThreads, 0, s>>>(m->theta16, m->theta, m->n_store);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_begin_call(ModelState* st, uint32_t budget, cudaStream_t s) {
  {
    ProfScope ps_("begin_call", s);
    k_begin_call<<<1, 1, 0, s>>>(st, budget);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_minmax(const float* vol, int64_t n, ModelState* st, cudaStream_t s) {
  DVNR_CUDA(cudaMemsetAsync(&st->enc_min, 0xFF, sizeof(uint32_t), s));
  DVNR_CUDA(cudaMemsetAsync(&st->enc_max, 0x00, sizeof(uint32_t), s));
  DVNR_CUDA(cudaMemsetAsync(&st->nonfinite, 0x00, sizeof(uint32_t), s));
  {
    ProfScope ps_("minmax", s);
    k_minmax<<<grid_for(n, kThreads), kThreads, 0, s>>>(vol, n, st);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_error_stats(const float* a, const float* b, int64_t n, double* out_dev,
                               cudaStream_t s) {
  DVNR_CUDA(cudaMemsetAsync(out_dev, 0, 2 * sizeof(double), s));
  {
    ProfScope ps_("error_stats", s);
    if (n > 0) k_error_stats<<<grid_for(n, kThreads), kThreads, 0, s>>>(a, b, n, out_dev);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_corner_indices(dvnr_model m, const uint32_t* coords, int64_t n, uint32_t* idx,
                                  cudaStream_t s) {
  {
    ProfScope ps_("corner_indices", s);
    if (n > 0) k_corner_indices<<<grid_for(n, kThreads), kThreads, 0, s>>>(m->lv, coords, n, idx);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status launch_adam(const AdamModelPtrs* models_dev, int n_models, int64_t n_params,
                        const AdamHyper& h, cudaStream_t s) {
  // ~4 blocks of 256 threads per SM over all models
  int per_model = (int)((152 * 8 + n_models - 1) / n_models);
  const int64_t need = (n_params / 4 + kThreads - 1) / kThreads;
  if (per_model > need) per_model = (int)(need > 0 ? need : 1);
  dim3 grid(per_model, n_models);
  {
    ProfScope ps_("adam", s);
    k_adam<<<grid, kThreads, 0, s>>>(models_dev, n_params, h);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

}  // namespace dvnr

// ---------------------------------------------------------------------------
// Allocation-free FP64 error statistics.
//
// For callers that must not allocate device memory when they ask for the
// error -- for example an in situ pipeline whose simulation has reserved the
// device memory for itself, or a time step that must not pay the implicit
// device synchronisation of cudaMalloc/cudaFree. The scratch lives in a
// fixed file-scope device array: one (sum, max) pair per block of
// kErrChunk elements, plus the final pair. Every GPU that loads the
// library holds it (64 KiB + 16 B) until the process exits.
namespace dvnr {
namespace {
constexpr int kErrBlocksMax = 4096;            // partial pairs in the scratch array
constexpr int64_t kErrChunk = 1 << 16;         // elements reduced by one block
constexpr int64_t kErrMaxN = (int64_t)kErrBlocksMax * kErrChunk;  // 2^28 elements
}  // namespace
}  // namespace dvnr

static __device__ __align__(256) double g_err_scratch[2 * dvnr::kErrBlocksMax + 2];

namespace dvnr {
namespace {

// Block b reduces elements [b kErrChunk, (b+1) kErrChunk) into part[2b],
// part[2b+1]; every pair of the launch is overwritten, so nothing has to be
// cleared between calls.
__global__ void __launch_bounds__(kThreads) k_error_partials(const float* __restrict__ a,
                                                            const float* __restrict__ b,
                                                            int64_t n, double* part) {
  const int64_t lo = (int64_t)blockIdx.x * kErrChunk;
  const int64_t hi = lo + kErrChunk < n ? lo + kErrChunk : n;
  double s = 0.0, mx = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double d = (double)__ldg(a + i) - (double)__ldg(b + i);
    s += d * d;
    mx = fmax(mx, fabs(d));
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double ss[kThreads / 32], sm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, m = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t += ss[w];
      m = fmax(m, sm[w]);
    }
    part[2 * blockIdx.x] = t;
    part[2 * blockIdx.x + 1] = m;
  }
}

// One block folds the nb partial pairs (fixed order) into out[0], out[1].
__global__ void __launch_bounds__(kThreads) k_error_final(double* part, int nb, double* out) {
  double s = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s += part[2 * i];
    mx = fmax(mx, part[2 * i + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double ss[kThreads / 32], sm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sm[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, m = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t += ss[w];
      m = fmax(m, sm[w]);
    }
    out[0] = t;
    out[1] = m;
  }
}

// Device address of g_err_scratch per device, looked up once per device
// (with that device current) on its first call.
constexpr int kMaxDevices = 64;
double* g_err_scratch_ptr[kMaxDevices] = {};
std::mutex g_err_scratch_mu;

dvnr_status err_scratch(double** out) {
  int dev = 0;
  DVNR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the %d devices this call supports", dev, kMaxDevices);
    return DVNR_E_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_err_scratch_mu);
  if (!g_err_scratch_ptr[dev]) {
    void* p = nullptr;
    DVNR_CUDA(cudaGetSymbolAddress(&p, g_err_scratch));
    g_err_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_err_scratch_ptr[dev];
  return DVNR_OK;
}

}  // namespace

// Resolve the scratch address of the current device ahead of the first
// dvnr_error_stats_noalloc call there (dvnr_create calls this), so that the
// lookup, and the module load it may trigger, happens outside that call.
dvnr_status prime_err_scratch() {
  double* p = nullptr;
  return err_scratch(&p);
}

}  // namespace dvnr

extern "C" dvnr_status dvnr_error_stats_noalloc(const float* a_dev, const float* b_dev, int64_t n,
                                                double* out_host, void* stream) {
  using namespace dvnr;
  if (!out_host || n < 0 || (n > 0 && (!a_dev || !b_dev))) {
    set_error("bad argument");
    return DVNR_E_INVALID;
  }
  if (n > kErrMaxN) {
    set_error("n = %lld exceeds the %lld elements the static scratch of dvnr_error_stats_noalloc "
              "can reduce",
              (long long)n, (long long)kErrMaxN);
    return DVNR_E_INVALID;
  }
  if (n == 0) {
    out_host[0] = 0.0;
    out_host[1] = 0.0;
    return DVNR_OK;
  }
  double* scratch = nullptr;
  dvnr_status rc = err_scratch(&scratch);
  if (rc != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)((n + kErrChunk - 1) / kErrChunk);
  double* fin = scratch + 2 * kErrBlocksMax;
  {
    ProfScope ps("error_stats_noalloc", s);
    k_error_partials<<<nb, kThreads, 0, s>>>(a_dev, b_dev, n, scratch);
  }
  DVNR_CUDA(cudaGetLastError());
  {
    ProfScope ps("error_stats_noalloc", s);
    k_error_final<<<1, kThreads, 0, s>>>(scratch, nb, fin);
  }
  DVNR_CUDA(cudaGetLastError());
  DVNR_CUDA(cudaMemcpyAsync(out_host, fin, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  DVNR_CUDA(cudaStreamSynchronize(s));
  return DVNR_OK;
}
