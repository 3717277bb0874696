// api.cu -- host implementation of the libdvnr C ABI (include/dvnr.h).
//
// Model lifecycle, argument checks, the per-step orchestration of the plain
// FP32 path and of the grouped FP16 tensor-core path (CUDA-graph replay),
// decoding and rendering. Every call returns a status and never aborts.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <vector>

#include "dvnr_internal.cuh"
#include "mp_path.cuh"

namespace dvnr {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

dvnr_status cuda_status(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? DVNR_E_OOM : DVNR_E_CUDA;
}

// Same encoding and MLP configuration: one FP16 grouped launch can hold them.
bool same_arch(const dvnr_model a, const dvnr_model b) {
  return a->enc.n_levels == b->enc.n_levels && a->enc.n_features == b->enc.n_features &&
         a->enc.log2_T == b->enc.log2_T && a->enc.base_res == b->enc.base_res &&
         a->enc.growth == b->enc.growth && a->mlp.width == b->mlp.width &&
         a->mlp.n_hidden == b->mlp.n_hidden;
}

namespace {

dvnr_status fail(dvnr_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

std::atomic<uint64_t> g_next_uid{1};

// Half-normal quantile table in 24-bit fixed point (Sec. 3.3 boundary
// samples): knot k < 4096 at p = k/4096, the last knot at p = 1 - 2^-24,
// q(p) = sigma sqrt(2) erfinv(p); erfinv by safeguarded Newton steps on erf.
double erfinv_newton(double p) {
  if (p <= 0.0) return 0.0;
  double lo = 0.0, hi = 8.0, x = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double f = std::erf(x) - p;
    if (f < 0.0) lo = x; else hi = x;
    const double d = 1.1283791670955126 * std::exp(-x * x);
    double xn = x - f / d;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (xn == x || hi - lo <= 0.0) break;
    x = xn;
  }
  return x;
}

void quantile_table(float sigma_f, std::vector<int32_t>& tab) {
  const double sigma = (double)sigma_f;
  tab.resize(kQTab + 1);
  for (int k = 0; k <= kQTab; ++k) {
    const double p = (k < kQTab) ? (double)k / kQTab : 1.0 - std::ldexp(1.0, -24);
    const double x = (k == 0) ? 0.0 : erfinv_newton(p);
    const double q = sigma * (1.41421356237309504880 * x);
    tab[k] = (int32_t)std::llround(q * 16777216.0);
  }
}

dvnr_status check_enc_mlp(const dvnr_enc_cfg* enc, const dvnr_mlp_cfg* mlp) {
  if (!enc || !mlp) return fail(DVNR_E_INVALID, "NULL configuration");
  if (enc->n_levels < 1 || enc->n_levels > kMaxLevels)
    return fail(DVNR_E_INVALID, "n_levels must be in [1, %d]", kMaxLevels);
  const int F = enc->n_features;
  if (!(F == 1 || F == 2 || F == 4 || F == 8))
    return fail(DVNR_E_INVALID, "n_features must be 1, 2, 4 or 8");
  if (enc->log2_T < 4 || enc->log2_T > 24) return fail(DVNR_E_INVALID, "log2_T must be in [4, 24]");
  if (enc->base_res < 1 || !(enc->growth >= 1.0) || !std::isfinite(enc->growth))
    return fail(DVNR_E_INVALID, "base_res >= 1 and finite growth >= 1 required");
  if (!(mlp->width == 16 || mlp->width == 32 || mlp->width == 64))
    return fail(DVNR_E_UNSUPPORTED, "width must be 16, 32 or 64");
  if (mlp->n_hidden < 1 || mlp->n_hidden > kMaxHidden)
    return fail(DVNR_E_INVALID, "n_hidden must be in [1, %d]", kMaxHidden);
  if (enc->n_levels * F > 256) return fail(DVNR_E_UNSUPPORTED, "n_levels * n_features > 256");
  return DVNR_OK;
}


dvnr_status check_train_cfg(const dvnr_train_cfg* c) {
  if (!c) return fail(DVNR_E_INVALID, "NULL train configuration");
  if (c->batch < 1) return fail(DVNR_E_INVALID, "batch must be >= 1");
  if (c->steps < 0) return fail(DVNR_E_INVALID, "steps must be >= 0");
  if (!(c->lr > 0.f) || !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
      !(c->eps >= 0.f) || !(c->weight_decay >= 0.f))
    return fail(DVNR_E_INVALID, "Adam hyper-parameters out of range");
  if (!(c->lambda_bnd >= 0.f && c->lambda_bnd <= 1.f))
    return fail(DVNR_E_INVALID, "lambda_bnd must be in [0, 1]");
  if (c->lambda_bnd > 0.f && !(c->sigma_bnd > 0.f && c->sigma_bnd <= 1.f))
    return fail(DVNR_E_INVALID, "sigma_bnd must be in (0, 1]");
  if (c->precision != DVNR_FP32 && c->precision != DVNR_FP16)
    return fail(DVNR_E_INVALID, "precision must be DVNR_FP32 or DVNR_FP16");
  if (c->loss != DVNR_LOSS_L1 && c->loss != DVNR_LOSS_L2)
    return fail(DVNR_E_INVALID, "loss must be DVNR_LOSS_L1 or DVNR_LOSS_L2");
  if (c->precision == DVNR_FP16 && c->growth_interval < 1)
    return fail(DVNR_E_INVALID, "growth_interval must be >= 1");
  if (c->epochs < 0 || c->min_steps < 0) return fail(DVNR_E_INVALID, "epochs and min_steps must be >= 0");
  if (!(c->stop_loss >= 0.f) || !std::isfinite(c->stop_loss))
    return fail(DVNR_E_INVALID, "stop_loss must be finite and >= 0");
  if (!(c->stop_decay >= 0.f && c->stop_decay < 1.f)) return fail(DVNR_E_INVALID, "stop_decay must be in [0, 1)");
  return DVNR_OK;
}

// Iterations of one training call for model m (Sec. 3.2):
// N_train^max = max(N_train^min, N_train), where N_train is the fixed count
// `steps`, or ceil(N_vox / N_batch) * N_epoch (N_vox the owned voxels of the
// partition) when epochs > 0.
int64_t train_budget(const dvnr_model m, const dvnr_train_cfg* c) {
  int64_t n = c->steps;
  if (c->epochs > 0) {
    const int64_t nvox = (m->box.hi[0] - m->box.lo[0]) * (m->box.hi[1] - m->box.lo[1]) *
                         (m->box.hi[2] - m->box.lo[2]);
    const int64_t per_epoch = (nvox + c->batch - 1) / c->batch;
    n = per_epoch > INT64_MAX / c->epochs ? INT64_MAX : per_epoch * c->epochs;
  }
  return std::max(c->min_steps, n);
}

dvnr_status use_device(dvnr_model m) {
  int cur = -1;
  DVNR_CUDA(cudaGetDevice(&cur));
  if (cur != m->device) DVNR_CUDA(cudaSetDevice(m->device));
  return DVNR_OK;
}

int64_t stored_voxels(const dvnr_model m) { return m->dims[0] * m->dims[1] * m->dims[2]; }

float initial_loss_scale(int32_t batch) {
  // 2^round(log2 B): the scaled L1 output gradient S/B is then ~1
  return std::ldexp(1.0f, (int)std::lround(std::log2((double)batch)));
}

dvnr_status prepare_qtab(dvnr_model m, float sigma, cudaStream_t s) {
  if (m->qtab_sigma == sigma) return DVNR_OK;
  std::vector<int32_t> tab;
  quantile_table(sigma > 0.f ? sigma : 0.005f, tab);
  DVNR_CUDA(cudaMemcpyAsync(m->qtab, tab.data(), tab.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  DVNR_CUDA(cudaStreamSynchronize(s));  // the host table is released below
  m->qtab_sigma = sigma;
  return DVNR_OK;
}

SampleParams sample_params(dvnr_model m, const dvnr_train_cfg* cfg, uint32_t slot) {
  SampleParams sp;
  sp.key = make_uint2((uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32));
  sp.model = slot;
  sp.n_bnd = (int32_t)std::floor((double)cfg->lambda_bnd * (double)cfg->batch);
  sp.qtab = m->qtab;
  return sp;
}

AdamHyper adam_hyper(const dvnr_train_cfg* cfg, bool mixed) {
  AdamHyper h;
  h.lr = cfg->lr;
  h.beta1 = cfg->beta1;
  h.beta2 = cfg->beta2;
  h.eps = cfg->eps;
  h.weight_decay = cfg->weight_decay;
  h.inv_batch = 1.0f / (float)cfg->batch;
  h.mixed = mixed ? 1 : 0;
  h.growth_interval = cfg->growth_interval > 0 ? cfg->growth_interval : (1 << 30);
  h.gated = 1;
  h.stop_loss = cfg->stop_loss;
  h.stop_decay = cfg->stop_decay;
  h.external = 0;
  h.dry = 0;
  return h;
}

// Per-model AdamModelPtrs live at the end of the model block.
AdamModelPtrs* adam_ptrs_dev(dvnr_model m) {
  return reinterpret_cast<AdamModelPtrs*>(reinterpret_cast<char*>(m->qtab) +
                                          align256((kQTab + 1) * sizeof(int32_t)));
}

}  // namespace
}  // namespace dvnr

using namespace dvnr;

extern "C" {

int32_t dvnr_abi_version(void) { return DVNR_ABI_VERSION; }

const char* dvnr_last_error(void) { return g_err; }

dvnr_status dvnr_create(const dvnr_box* box, const dvnr_enc_cfg* enc, const dvnr_mlp_cfg* mlp,
                        uint64_t seed, dvnr_model* out) {
  dvnr::ApiRange nvtx_("dvnr_create");
  g_err[0] = 0;
  if (!out) return fail(DVNR_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!box) return fail(DVNR_E_INVALID, "box is NULL");
  dvnr_status rc = check_enc_mlp(enc, mlp);
  if (rc != DVNR_OK) return rc;
  if (box->ghost < 0) return fail(DVNR_E_INVALID, "ghost must be >= 0");
  int64_t dims[3];
  for (int a = 0; a < 3; ++a) {
    if (box->hi[a] <= box->lo[a]) return fail(DVNR_E_INVALID, "box must have hi > lo on every axis");
    dims[a] = box->hi[a] - box->lo[a] + 2 * (int64_t)box->ghost;
    if (dims[a] < 2) return fail(DVNR_E_INVALID, "stored block needs >= 2 voxels per axis");
    if (dims[a] > (1 << 20)) return fail(DVNR_E_INVALID, "block too large");
  }
  dvnr_model m = new (std::nothrow) dvnr_model_s();
  if (!m) return fail(DVNR_E_OOM, "host allocation failed");
  m->uid = g_next_uid.fetch_add(1);
  m->box = *box;
  m->enc = *enc;
  m->mlp = *mlp;
  for (int a = 0; a < 3; ++a) m->dims[a] = dims[a];
  cudaError_t ce = cudaGetDevice(&m->device);
  if (ce != cudaSuccess) {
    delete m;
    return cuda_status(ce, "cudaGetDevice");
  }
  // Level layout: N_l = floor(base growth^l); dense iff (N_l + 1)^3 <= T.
  LevelTab& lv = m->lv;
  lv.L = enc->n_levels;
  lv.F = enc->n_features;
  lv.in_dim = enc->n_levels * enc->n_features;
  const int64_t T = 1LL << enc->log2_T;
  lv.hash_mask = (uint32_t)(T - 1);
  lv.dense_mask = 0;
  int64_t off = 0, ext = 0;
  auto padded = [](int64_t v) { return (v + kParamAlign - 1) / kParamAlign * kParamAlign; };
  m->lmap.L = lv.L;
  for (int l = 0; l < lv.L; ++l) {
    const double r = std::floor((double)enc->base_res * std::pow(enc->growth, (double)l));
    if (r > (double)(1 << 21)) {
      delete m;
      return fail(DVNR_E_INVALID, "level %d resolution exceeds 2^21", l);
    }
    const int64_t N = (int64_t)r;
    lv.N[l] = (uint32_t)N;
    const int64_t verts = (N + 1) * (N + 1) * (N + 1);
    const bool dense = verts <= T;
    if (dense) lv.dense_mask |= 1u << l;
    lv.off[l] = off;
    m->lmap.int_off[l] = off;
    m->lmap.ext_off[l] = ext;
    const int64_t len = (dense ? verts : T) * lv.F;
    off = padded(off + len);
    ext += len;
  }
  m->n_enc = ext;
  m->lmap.ext_off[lv.L] = ext;
  m->lmap.int_off[lv.L] = off;
  int64_t w = off;
  const int W = mlp->width, H = mlp->n_hidden;
  for (int k = 0; k < H; ++k) {
    const int fan_in = k == 0 ? lv.in_dim : W;
    m->w_off[k] = w;
    m->glorot[k] = std::sqrt(6.0 / (double)(fan_in + W));
    w += (int64_t)W * fan_in;
  }
  m->w_off[H] = w;
  m->glorot[H] = std::sqrt(6.0 / (double)(W + 1));
  w += W;
  m->n_mlp = w - off;
  m->n_params = m->n_enc + m->n_mlp;
  m->lmap.ext_off[lv.L + 1] = m->n_params;
  m->n_store = padded(w);
  if (m->n_store >= (1LL << 31)) {
    delete m;
    return fail(DVNR_E_UNSUPPORTED, "more than 2^31 parameters");
  }
  const size_t P = (size_t)m->n_store;
  const size_t b32 = align256(P * 4), b16 = align256(P * 2), bst = align256(sizeof(ModelState)),
               bq = align256((kQTab + 1) * sizeof(int32_t)), bap = align256(sizeof(AdamModelPtrs));
  m->block_bytes = 4 * b32 + b16 + bst + bq + bap;
  ce = dev_malloc(reinterpret_cast<void**>(&m->block), m->block_bytes);
  if (ce != cudaSuccess) {
    delete m;
    return cuda_status(ce, "cudaMalloc(model)");
  }
  char* p = static_cast<char*>(m->block);
  m->theta = reinterpret_cast<float*>(p); p += b32;
  m->m1 = reinterpret_cast<float*>(p); p += b32;
  m->m2 = reinterpret_cast<float*>(p); p += b32;
  m->grad = reinterpret_cast<float*>(p); p += b32;
  m->theta16 = reinterpret_cast<__half*>(p); p += b16;
  m->st = reinterpret_cast<ModelState*>(p); p += bst;
  m->qtab = reinterpret_cast<int32_t*>(p); p += bq;
  AdamModelPtrs ap{m->theta, m->m1, m->m2, m->grad, m->theta16, m->st};
  ModelState st0{};
  st0.enc_min = float_to_ordered(0.f);
  st0.enc_max = float_to_ordered(1.f);
  st0.loss_scale = 1.f;
  auto cleanup = [&](dvnr_status s) {
    dev_free(m->block);
    delete m;
    return s;
  };
  if ((ce = cudaMemset(m->m1, 0, 3 * b32)) != cudaSuccess) return cleanup(cuda_status(ce, "cudaMemset"));
  // storage padding between level tables stays zero in theta and its FP16 copy
  if ((ce = cudaMemset(m->theta, 0, b32)) != cudaSuccess ||
      (ce = cudaMemset(m->theta16, 0, b16)) != cudaSuccess)
    return cleanup(cuda_status(ce, "cudaMemset"));
  if ((rc = launch_init_params(m, seed, 0)) != DVNR_OK) return cleanup(rc);
  if ((rc = prime_err_scratch()) != DVNR_OK) return cleanup(rc);
  if ((ce = cudaMemcpy(m->st, &st0, sizeof(st0), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(adam_ptrs_dev(m), &ap, sizeof(ap), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaDeviceSynchronize()) != cudaSuccess)
    return cleanup(cuda_status(ce, "dvnr_create"));
  *out = m;
  return DVNR_OK;
}

void dvnr_destroy(dvnr_model m) {
  if (!m) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  mp_release(m);
  if (m->ws.base) dev_free(m->ws.base);
  if (m->grid_ws) dev_free(m->grid_ws);
  dev_free(m->block);
  if (cur >= 0) cudaSetDevice(cur);
  delete m;
}

dvnr_status dvnr_freeze(dvnr_model m, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_freeze");
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (m->frozen) return DVNR_OK;
  if (!mp_supported(m)) return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if ((rc = launch_refresh_half(m, (cudaStream_t)stream)) != DVNR_OK) return rc;
  const size_t b16 = align256((size_t)m->n_store * 2), bst = align256(sizeof(ModelState));
  void* blk = nullptr;
  DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&blk), b16 + bst));
  char* p = static_cast<char*>(blk);
  cudaError_t e = cudaMemcpyAsync(p, m->theta16, (size_t)m->n_store * 2, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p + b16, m->st, sizeof(ModelState), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    dev_free(blk);
    return cuda_status(e, "dvnr_freeze");
  }
  mp_release(m);
  if (m->ws.base) dev_free(m->ws.base);
  m->ws = Fp32Workspace{};
  if (m->grid_ws) dev_free(m->grid_ws);
  m->grid_ws = nullptr;
  m->grid_ws_elems = 0;
  dev_free(m->block);
  m->block = blk;
  m->block_bytes = b16 + bst;
  m->theta = m->m1 = m->m2 = m->grad = nullptr;
  m->qtab = nullptr;
  m->qtab_sigma = -1.f;
  m->theta16 = reinterpret_cast<__half*>(p);
  m->st = reinterpret_cast<ModelState*>(p + b16);
  m->precision = DVNR_FP16;
  m->frozen = true;
  return DVNR_OK;
}

dvnr_status dvnr_param_count(dvnr_model m, int64_t* n_enc, int64_t* n_mlp) {
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (n_enc) *n_enc = m->n_enc;
  if (n_mlp) *n_mlp = m->n_mlp;
  return DVNR_OK;
}

namespace dvnr {
namespace {
// Copy between the compact host layout and storage, block by block.
dvnr_status copy_blocks(dvnr_model m, float* host, const float* host_src, bool to_host) {
  for (int b = 0; b <= m->lmap.L; ++b) {
    const int64_t e0 = m->lmap.ext_off[b], len = m->lmap.ext_off[b + 1] - e0;
    const int64_t i0 = m->lmap.int_off[b];
    if (to_host)
      DVNR_CUDA(cudaMemcpy(host + e0, m->theta + i0, (size_t)len * 4, cudaMemcpyDeviceToHost));
    else
      DVNR_CUDA(cudaMemcpy(m->theta + i0, host_src + e0, (size_t)len * 4, cudaMemcpyHostToDevice));
  }
  return DVNR_OK;
}
}  // namespace
}  // namespace dvnr

dvnr_status dvnr_adaptive_encoding(int64_t n_vox, int64_t n_vox_global, int32_t log2_T_ref,
                                   int32_t log2_T_min, double R_ref, dvnr_enc_cfg* enc) {
  if (!enc) return fail(DVNR_E_INVALID, "NULL encoding configuration");
  if (n_vox < 1 || n_vox > n_vox_global) return fail(DVNR_E_INVALID, "need 1 <= n_vox <= n_vox_global");
  if (log2_T_min < 1 || log2_T_min > log2_T_ref || log2_T_ref > 31)
    return fail(DVNR_E_INVALID, "need 1 <= log2_T_min <= log2_T_ref <= 31");
  if (!(R_ref >= 1.0) || !std::isfinite(R_ref)) return fail(DVNR_E_INVALID, "R_ref must be finite and >= 1");
  // T = 2^k with k the smallest exponent such that 2^k n_global >= T_ref n_vox
  const unsigned __int128 want = (unsigned __int128)(uint64_t)n_vox << log2_T_ref;
  int k = 0;
  while (((unsigned __int128)(uint64_t)n_vox_global << k) < want) ++k;
  k = std::max(k, (int)log2_T_min);
  // R_0: the largest R with R^3 T_ref <= R_ref^3 T (exact when R_ref is an
  // integer), else from the cube root
  int64_t r;
  const int e = k - log2_T_ref;  // <= 0 since n_vox <= n_vox_global
  if (R_ref == std::floor(R_ref) && R_ref < 1e6) {
    const unsigned __int128 rr = (unsigned __int128)(uint64_t)R_ref;
    const unsigned __int128 rhs = rr * rr * rr;  // R_ref^3, compared as R^3 2^-e <= R_ref^3
    r = (int64_t)R_ref;
    while (r > 1 && (((unsigned __int128)r * r * r) << (-e)) > rhs) --r;
  } else {
    r = (int64_t)std::floor(R_ref * std::cbrt(std::ldexp(1.0, e)));
  }
  enc->log2_T = k;
  enc->base_res = (int32_t)std::max<int64_t>(1, r);
  return DVNR_OK;
}

dvnr_status dvnr_export_fp16(dvnr_model m, uint16_t* host, int64_t n) {
  if (!m || !host) return fail(DVNR_E_INVALID, "NULL argument");
  if (n != m->n_params) return fail(DVNR_E_INVALID, "n must equal n_enc + n_mlp = %lld", (long long)m->n_params);
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  if (!m->frozen && (rc = launch_refresh_half(m, 0)) != DVNR_OK) return rc;  // the copy follows the master weights
  DVNR_CUDA(cudaDeviceSynchronize());
  for (int b = 0; b <= m->lmap.L; ++b) {
    const int64_t e0 = m->lmap.ext_off[b], len = m->lmap.ext_off[b + 1] - e0;
    DVNR_CUDA(cudaMemcpy(host + e0, m->theta16 + m->lmap.int_off[b], (size_t)len * 2,
                         cudaMemcpyDeviceToHost));
  }
  return DVNR_OK;
}

dvnr_status dvnr_import_fp16(dvnr_model m, const uint16_t* host, int64_t n) {
  if (!m || !host) return fail(DVNR_E_INVALID, "NULL argument");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  if (n != m->n_params) return fail(DVNR_E_INVALID, "n must equal n_enc + n_mlp = %lld", (long long)m->n_params);
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  for (int b = 0; b <= m->lmap.L; ++b) {
    const int64_t e0 = m->lmap.ext_off[b], len = m->lmap.ext_off[b + 1] - e0;
    DVNR_CUDA(cudaMemcpy(m->theta16 + m->lmap.int_off[b], host + e0, (size_t)len * 2,
                         cudaMemcpyHostToDevice));
  }
  if ((rc = launch_widen_half(m, 0)) != DVNR_OK) return rc;
  DVNR_CUDA(cudaMemset(m->m1, 0, (size_t)m->n_store * 4));
  DVNR_CUDA(cudaMemset(m->m2, 0, (size_t)m->n_store * 4));
  DVNR_CUDA(cudaMemset(m->grad, 0, (size_t)m->n_store * 4));
  if ((rc = launch_state_reset(m->st, 1.f, 0)) != DVNR_OK) return rc;
  m->scale_initialized = false;
  DVNR_CUDA(cudaDeviceSynchronize());
  return DVNR_OK;
}

dvnr_status dvnr_get_weights(dvnr_model m, float* host, int64_t n) {
  if (!m || !host) return fail(DVNR_E_INVALID, "NULL argument");
  if (n != m->n_params) return fail(DVNR_E_INVALID, "n must equal n_enc + n_mlp = %lld", (long long)m->n_params);
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  if (m->frozen) {  // the FP16 parameters, widened
    std::vector<uint16_t> h16((size_t)n);
    if ((rc = dvnr_export_fp16(m, h16.data(), n)) != DVNR_OK) return rc;
    for (int64_t i = 0; i < n; ++i) host[i] = __half2float(__ushort_as_half(h16[(size_t)i]));
    return DVNR_OK;
  }
  return copy_blocks(m, host, nullptr, true);
}

dvnr_status dvnr_set_weights(dvnr_model m, const float* host, int64_t n) {
  if (!m || !host) return fail(DVNR_E_INVALID, "NULL argument");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  if (n != m->n_params) return fail(DVNR_E_INVALID, "n must equal n_enc + n_mlp = %lld", (long long)m->n_params);
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  if ((rc = copy_blocks(m, nullptr, host, false)) != DVNR_OK) return rc;
  if ((rc = launch_refresh_half(m, 0)) != DVNR_OK) return rc;
  DVNR_CUDA(cudaMemset(m->m1, 0, (size_t)m->n_store * 4));
  DVNR_CUDA(cudaMemset(m->m2, 0, (size_t)m->n_store * 4));
  DVNR_CUDA(cudaMemset(m->grad, 0, (size_t)m->n_store * 4));
  if ((rc = launch_state_reset(m->st, 1.f, 0)) != DVNR_OK) return rc;
  m->scale_initialized = false;
  DVNR_CUDA(cudaDeviceSynchronize());
  return DVNR_OK;
}

dvnr_status dvnr_copy_weights(dvnr_model dst, dvnr_model src, void* stream) {
  if (!dst || !src) return fail(DVNR_E_INVALID, "NULL model");
  if (!same_arch(dst, src)) return fail(DVNR_E_INVALID, "models differ in encoding or MLP configuration");
  if (dst->device != src->device) return fail(DVNR_E_INVALID, "models live on different devices");
  if (dst->frozen) return fail(DVNR_E_STATE, "the destination model is frozen");
  if (dst == src) return DVNR_OK;
  dvnr_status rc = use_device(dst);
  if (rc != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)dst->n_store;
  DVNR_CUDA(cudaMemcpyAsync(dst->theta16, src->theta16, n * 2, cudaMemcpyDeviceToDevice, s));
  if (src->frozen) {  // a frozen source has only its FP16 parameters: widen them
    if ((rc = launch_widen_half(dst, s)) != DVNR_OK) return rc;
  } else {
    DVNR_CUDA(cudaMemcpyAsync(dst->theta, src->theta, n * 4, cudaMemcpyDeviceToDevice, s));
  }
  DVNR_CUDA(cudaMemcpyAsync(dst->st, src->st, 2 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  DVNR_CUDA(cudaMemsetAsync(dst->m1, 0, n * 4, s));
  DVNR_CUDA(cudaMemsetAsync(dst->m2, 0, n * 4, s));
  DVNR_CUDA(cudaMemsetAsync(dst->grad, 0, n * 4, s));
  if ((rc = launch_state_reset(dst->st, 1.f, s)) != DVNR_OK) return rc;
  dst->precision = src->precision;
  dst->scale_initialized = false;
  return DVNR_OK;
}

dvnr_status dvnr_set_precision(dvnr_model m, int32_t precision, void* stream) {
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (precision != DVNR_FP32 && precision != DVNR_FP16) return fail(DVNR_E_INVALID, "bad precision");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  if (m->frozen && precision != DVNR_FP16) return fail(DVNR_E_STATE, "a frozen model decodes in FP16 only");
  if (precision == DVNR_FP16 && m->precision != DVNR_FP16) {
    if (!mp_supported(m)) return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
    if ((rc = launch_refresh_half(m, (cudaStream_t)stream)) != DVNR_OK) return rc;
  }
  m->precision = precision;
  return DVNR_OK;
}

dvnr_status dvnr_get_state(dvnr_model m, dvnr_state_info* out) {
  if (!m || !out) return fail(DVNR_E_INVALID, "NULL argument");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  ModelState st;
  DVNR_CUDA(cudaMemcpy(&st, m->st, sizeof(st), cudaMemcpyDeviceToHost));
  out->vmin = ordered_to_float(st.enc_min);
  out->vmax = ordered_to_float(st.enc_max);
  out->loss_scale = st.loss_scale;
  out->last_loss = st.last_loss;
  out->iter = st.iter;
  out->adam_t = st.adam_t;
  out->skipped = st.skipped;
  out->n_enc = m->n_enc;
  out->n_mlp = m->n_mlp;
  out->precision = m->precision;
  out->nonfinite_input = st.nonfinite ? 1 : 0;
  out->loss_ema = st.loss_ema;
  out->budget_end = st.stop_at;
  out->stopped = st.stopped ? 1 : 0;
  out->frozen = m->frozen ? 1 : 0;
  if (st.timeouts) return fail(DVNR_E_TIMEOUT, "a bounded device wait gave up (%u)", st.timeouts);
  if (st.nonfinite) return fail(DVNR_E_NONFINITE_INPUT, "the last training volume held NaN/Inf");
  return DVNR_OK;
}

dvnr_status dvnr_set_value_range(dvnr_model m, double vmin, double vmax, void* stream) {
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (!std::isfinite(vmin) || !std::isfinite(vmax) || !(vmin <= vmax) ||
      !std::isfinite((float)vmin) || !std::isfinite((float)vmax))
    return fail(DVNR_E_INVALID, "value range needs finite vmin <= vmax");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  // enc_min and enc_max are adjacent words of the device state
  const uint32_t enc[2] = {float_to_ordered((float)vmin), float_to_ordered((float)vmax)};
  static_assert(offsetof(ModelState, enc_max) == offsetof(ModelState, enc_min) + sizeof(uint32_t),
                "value range words must be adjacent");
  cudaStream_t s = (cudaStream_t)stream;
  DVNR_CUDA(cudaMemcpyAsync(&m->st->enc_min, enc, sizeof(enc), cudaMemcpyHostToDevice, s));
  DVNR_CUDA(cudaStreamSynchronize(s));
  return DVNR_OK;
}

dvnr_status dvnr_train(dvnr_model* models, int32_t n, const float* const* vol_dev,
                       const dvnr_train_cfg* cfg, void* stream, float* final_loss_host) {
  dvnr::ApiRange nvtx_("dvnr_train");
  g_err[0] = 0;
  if (n < 1 || !models || !vol_dev) return fail(DVNR_E_INVALID, "need n >= 1 models and volumes");
  dvnr_status rc = check_train_cfg(cfg);
  if (rc != DVNR_OK) return rc;
  for (int i = 0; i < n; ++i) {
    if (!models[i] || !vol_dev[i]) return fail(DVNR_E_INVALID, "model or volume %d is NULL", i);
    if (models[i]->frozen) return fail(DVNR_E_STATE, "model %d is frozen", i);
    if (models[i]->device != models[0]->device) return fail(DVNR_E_INVALID, "models on different devices");
    for (int j = 0; j < i; ++j)
      if (models[j] == models[i]) return fail(DVNR_E_INVALID, "model %d appears twice", i);
  }
  const bool mixed = cfg->precision == DVNR_FP16;
  if (mixed) {
    for (int i = 0; i < n; ++i)
      if (!mp_supported(models[i]))
        return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  }
  std::vector<int64_t> budget((size_t)n);
  int64_t max_budget = 0;
  for (int i = 0; i < n; ++i) {
    budget[i] = train_budget(models[i], cfg);
    if (budget[i] > 0x7FFFFFFF) return fail(DVNR_E_INVALID, "model %d: iteration budget above 2^31 - 1", i);
    max_budget = std::max(max_budget, budget[i]);
  }
  if ((rc = use_device(models[0])) != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    dvnr_model m = models[i];
    if ((rc = launch_begin_call(m->st, (uint32_t)budget[i], s)) != DVNR_OK) return rc;
    if (cfg->lambda_bnd > 0.f && (rc = prepare_qtab(m, cfg->sigma_bnd, s)) != DVNR_OK) return rc;
    if ((rc = launch_minmax(vol_dev[i], stored_voxels(m), m->st, s)) != DVNR_OK) return rc;
    m->precision = cfg->precision;
    if (mixed && !m->scale_initialized) {
      if ((rc = launch_state_reset_scale(m->st, initial_loss_scale(cfg->batch), s)) != DVNR_OK) return rc;
      m->scale_initialized = true;
    }
  }
  const AdamHyper h = adam_hyper(cfg, mixed);
  if (mixed) {
    // one grouped launch per configuration class (models of a decomposition
    // with adaptive table sizes differ in T and R_0); each model keeps its
    // RNG slot, its index in this call
    std::vector<std::vector<int>> classes;
    for (int i = 0; i < n; ++i) {
      bool placed = false;
      for (auto& c : classes)
        if (same_arch(models[c[0]], models[i])) {
          c.push_back(i);
          placed = true;
          break;
        }
      if (!placed) classes.push_back({i});
    }
    for (const auto& c : classes) {
      std::vector<dvnr_model> cm;
      std::vector<const float*> cv;
      std::vector<uint32_t> slots;
      int64_t cmax = 0;
      for (int i : c) {
        cm.push_back(models[i]);
        cv.push_back(vol_dev[i]);
        slots.push_back((uint32_t)i);
        cmax = std::max(cmax, budget[i]);
      }
      bool uniform = true;
      for (int i : c) uniform &= budget[i] == cmax;
      if (cmax > 0 && (rc = mp_train(cm.data(), (int)c.size(), cv.data(), slots.data(), cfg, h, cmax,
                                     uniform, s)) != DVNR_OK)
        return rc;
    }
  } else {
    for (int i = 0; i < n; ++i) {
      dvnr_model m = models[i];
      if ((rc = fp32_ensure_workspace(m, cfg->batch)) != DVNR_OK) return rc;
      Fp32StepArgs a{};
      a.m = m;
      a.vol = vol_dev[i];
      a.sp = sample_params(m, cfg, (uint32_t)i);
      a.batch = cfg->batch;
      a.loss = cfg->loss;
      a.explicit_iter = false;
      a.gated = true;
      // the kernels of a step do nothing once the model stopped early
      for (int64_t step = 0; step < budget[i]; ++step) {
        if ((rc = fp32_forward_backward(a, s)) != DVNR_OK) return rc;
        if ((rc = launch_adam(adam_ptrs_dev(m), 1, m->n_store, h, s)) != DVNR_OK) return rc;
      }
    }
  }
  if (final_loss_host) {
    DVNR_CUDA(cudaStreamSynchronize(s));
    bool bad = false;
    for (int i = 0; i < n; ++i) {
      ModelState st;
      DVNR_CUDA(cudaMemcpy(&st, models[i]->st, sizeof(st), cudaMemcpyDeviceToHost));
      final_loss_host[i] = st.last_loss;
      bad |= st.nonfinite != 0;
      if (st.timeouts) return fail(DVNR_E_TIMEOUT, "a bounded device wait gave up in model %d", i);
    }
    if (bad) return fail(DVNR_E_NONFINITE_INPUT, "a training volume held NaN/Inf");
  }
  return DVNR_OK;
}

dvnr_status dvnr_train_grad(dvnr_model m, const float* vol_dev, const dvnr_train_cfg* cfg,
                            int64_t iteration, const dvnr_step_outputs* out, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_train_grad");
  g_err[0] = 0;
  if (!m || !vol_dev) return fail(DVNR_E_INVALID, "NULL model or volume");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  dvnr_status rc = check_train_cfg(cfg);
  if (rc != DVNR_OK) return rc;
  if (iteration < 0) return fail(DVNR_E_INVALID, "iteration must be >= 0");
  const bool mixed = cfg->precision == DVNR_FP16;
  if (mixed && !mp_supported(m))
    return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  if ((rc = use_device(m)) != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  dvnr_step_outputs o{};
  if (out) o = *out;
  if (cfg->lambda_bnd > 0.f && (rc = prepare_qtab(m, cfg->sigma_bnd, s)) != DVNR_OK) return rc;
  if ((rc = launch_minmax(vol_dev, stored_voxels(m), m->st, s)) != DVNR_OK) return rc;
  DVNR_CUDA(cudaMemsetAsync(&m->st->loss_sum, 0, sizeof(float), s));
  float S = 1.f;
  if (mixed) {
    S = initial_loss_scale(cfg->batch);
    MpStepDebug dbg{o.y, o.dx0, o.target, o.coords};
    rc = mp_train_grad(m, vol_dev, cfg, (uint32_t)iteration, S, dbg, s);
  } else {
    Fp32StepArgs a{};
    a.m = m;
    a.vol = vol_dev;
    a.sp = sample_params(m, cfg, 0);
    a.batch = cfg->batch;
    a.loss = cfg->loss;
    a.explicit_iter = true;
    a.iter = (uint32_t)iteration;
    a.y_out = o.y;
    a.dx0_out = o.dx0;
    a.tgt_out = o.target;
    a.coords_out = o.coords;
    rc = fp32_forward_backward(a, s);
  }
  if (rc != DVNR_OK) return rc;
  return launch_finish_grad(m, S, 1.0f / (float)cfg->batch, o.grad, o.loss, s);
}

dvnr_status dvnr_adam_step(dvnr_model m, const float* grad_dev, const dvnr_train_cfg* cfg,
                           void* stream) {
  dvnr::ApiRange nvtx_("dvnr_adam_step");
  g_err[0] = 0;
  if (!m || !grad_dev) return fail(DVNR_E_INVALID, "NULL model or gradient");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  dvnr_status rc = check_train_cfg(cfg);
  if (rc != DVNR_OK) return rc;
  const bool mixed = cfg->precision == DVNR_FP16;
  if (mixed && !mp_supported(m))
    return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  if ((rc = use_device(m)) != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (mixed && !m->scale_initialized) {
    if ((rc = launch_state_reset_scale(m->st, initial_loss_scale(cfg->batch), s)) != DVNR_OK) return rc;
    m->scale_initialized = true;
  }
  if ((rc = launch_load_grad(m, grad_dev, mixed, s)) != DVNR_OK) return rc;
  AdamHyper h = adam_hyper(cfg, mixed);
  h.gated = 0;  // not bound to a training call's budget
  h.external = 1;
  h.stop_loss = 0.f;
  if ((rc = launch_adam(adam_ptrs_dev(m), 1, m->n_store, h, s)) != DVNR_OK) return rc;
  m->precision = cfg->precision;
  return DVNR_OK;
}

dvnr_status dvnr_load_params(dvnr_model m, const float* params_dev, void* stream) {
  if (!m || !params_dev) return fail(DVNR_E_INVALID, "NULL model or parameters");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  return launch_load_params(m, params_dev, (cudaStream_t)stream);
}

dvnr_status dvnr_forward(dvnr_model m, const uint32_t* coords_dev, int64_t n, int32_t precision,
                         float* y_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_forward");
  g_err[0] = 0;
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (n < 0) return fail(DVNR_E_INVALID, "n must be >= 0");
  if (precision != DVNR_FP32 && precision != DVNR_FP16) return fail(DVNR_E_INVALID, "bad precision");
  if (n == 0) return DVNR_OK;
  if (!coords_dev || !y_dev) return fail(DVNR_E_INVALID, "NULL buffer");
  if (precision == DVNR_FP16 && !mp_supported(m))
    return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  if (precision == DVNR_FP32 && m->frozen) return fail(DVNR_E_STATE, "a frozen model keeps FP16 parameters only");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == DVNR_FP16) return mp_forward(m, coords_dev, n, y_dev, s);
  return fp32_decode_unit(m, coords_dev, nullptr, n, 0, y_dev, s, true);
}

dvnr_status dvnr_backward(dvnr_model m, const uint32_t* coords_dev, int64_t n, const float* dy_dev,
                          int32_t precision, float loss_scale, float* grad_dev, float* dx0_dev,
                          void* stream) {
  dvnr::ApiRange nvtx_("dvnr_backward");
  g_err[0] = 0;
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (m->frozen) return fail(DVNR_E_STATE, "the model is frozen");
  if (n < 1 || n > (1LL << 30)) return fail(DVNR_E_INVALID, "n must be in [1, 2^30]");
  if (precision != DVNR_FP32 && precision != DVNR_FP16) return fail(DVNR_E_INVALID, "bad precision");
  if (!coords_dev || !dy_dev || !grad_dev) return fail(DVNR_E_INVALID, "NULL buffer");
  if (!(loss_scale >= 0.f) || !std::isfinite(loss_scale)) return fail(DVNR_E_INVALID, "loss_scale must be finite and >= 0");
  const bool mixed = precision == DVNR_FP16;
  if (mixed && !mp_supported(m))
    return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (mixed) {
    if ((rc = launch_ext_scale(m, dy_dev, n, loss_scale, s)) != DVNR_OK) return rc;
    if ((rc = mp_backward(m, coords_dev, dy_dev, n, &m->st->ext_scale, dx0_dev, s)) != DVNR_OK) return rc;
    return launch_finish_grad_dev(m, &m->st->ext_scale, grad_dev, s);
  }
  Fp32StepArgs a{};
  a.m = m;
  a.vol = nullptr;
  a.batch = (int32_t)n;
  a.loss = DVNR_LOSS_L2;
  a.explicit_iter = true;
  a.gated = false;
  a.dx0_out = dx0_dev;
  a.ext_coords = coords_dev;
  a.ext_dy = dy_dev;
  if ((rc = fp32_forward_backward(a, s)) != DVNR_OK) return rc;
  return launch_finish_grad(m, 1.0f, 1.0f, grad_dev, nullptr, s);
}

dvnr_status dvnr_get_moments(dvnr_model m, float* m1_host, float* m2_host, int64_t n) {
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (m->frozen) return fail(DVNR_E_STATE, "a frozen model keeps no optimiser state");
  if (n != m->n_params) return fail(DVNR_E_INVALID, "n must equal n_enc + n_mlp = %lld", (long long)m->n_params);
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  DVNR_CUDA(cudaDeviceSynchronize());
  for (int b = 0; b <= m->lmap.L; ++b) {
    const int64_t e0 = m->lmap.ext_off[b], len = m->lmap.ext_off[b + 1] - e0;
    const int64_t i0 = m->lmap.int_off[b];
    if (m1_host)
      DVNR_CUDA(cudaMemcpy(m1_host + e0, m->m1 + i0, (size_t)len * 4, cudaMemcpyDeviceToHost));
    if (m2_host)
      DVNR_CUDA(cudaMemcpy(m2_host + e0, m->m2 + i0, (size_t)len * 4, cudaMemcpyDeviceToHost));
  }
  return DVNR_OK;
}

dvnr_status dvnr_decode_points(dvnr_model m, const float* xyz_dev, int64_t n, float* out_dev,
                               void* stream) {
  dvnr::ApiRange nvtx_("dvnr_decode_points");
  if (!m) return fail(DVNR_E_INVALID, "model is NULL");
  if (n < 0) return fail(DVNR_E_INVALID, "n must be >= 0");
  if (n == 0) return DVNR_OK;
  if (!xyz_dev || !out_dev) return fail(DVNR_E_INVALID, "NULL buffer");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  if (m->precision == DVNR_FP16) return mp_decode(m, xyz_dev, n, 0, out_dev, (cudaStream_t)stream);
  return fp32_decode_unit(m, nullptr, xyz_dev, n, 0, out_dev, (cudaStream_t)stream);
}

dvnr_status dvnr_decode_grid(dvnr_model m, float* out_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_decode_grid");
  if (!m || !out_dev) return fail(DVNR_E_INVALID, "NULL argument");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  const int64_t n = (m->box.hi[0] - m->box.lo[0]) * (m->box.hi[1] - m->box.lo[1]) *
                    (m->box.hi[2] - m->box.lo[2]);
  if (m->precision == DVNR_FP16) return mp_decode(m, nullptr, n, 1, out_dev, (cudaStream_t)stream);
  return fp32_decode_unit(m, nullptr, nullptr, n, 1, out_dev, (cudaStream_t)stream);
}

static dvnr_status check_render(const dvnr_model* models, int32_t n, const dvnr_tf* tf, int32_t w,
                                int32_t h, int32_t spr, float* rgba_dev) {
  if (n < 1 || !models || !tf || !rgba_dev) return fail(DVNR_E_INVALID, "NULL argument or n < 1");
  if (w < 1 || h < 1 || spr < 1) return fail(DVNR_E_INVALID, "w, h, spr must be >= 1");
  for (int i = 0; i < n; ++i) {
    if (!models[i]) return fail(DVNR_E_INVALID, "model %d is NULL", i);
    if (models[i]->device != models[0]->device) return fail(DVNR_E_INVALID, "models on different devices");
  }
  return DVNR_OK;
}

static void union_frame(const dvnr_model* models, int32_t n, float lo[3], float hi[3]) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = 1e30f;
    hi[a] = -1e30f;
    for (int i = 0; i < n; ++i) {
      lo[a] = std::min(lo[a], (float)models[i]->box.lo[a]);
      hi[a] = std::max(hi[a], (float)models[i]->box.hi[a]);
    }
  }
}

static dvnr_status render_grid(const dvnr_model* models, int32_t n, const float lo[3], const float hi[3],
                               const dvnr_tf* tf, int32_t w, int32_t h, int32_t spr, float* rgba_dev,
                               void* stream) {
  dvnr_status rc = use_device(models[0]);
  if (rc != DVNR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<RenderBlock> blocks((size_t)n);
  for (int i = 0; i < n; ++i) {
    dvnr_model m = models[i];
    const size_t ne = (size_t)((m->box.hi[0] - m->box.lo[0]) * (m->box.hi[1] - m->box.lo[1]) *
                               (m->box.hi[2] - m->box.lo[2]));
    if (m->grid_ws_elems < ne) {
      if (m->grid_ws) {
        DVNR_CUDA(cudaStreamSynchronize(s));
        dev_free(m->grid_ws);
        m->grid_ws = nullptr;
        m->grid_ws_elems = 0;
      }
      DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&m->grid_ws), ne * sizeof(float)));
      m->grid_ws_elems = ne;
    }
    if ((rc = dvnr_decode_grid(m, m->grid_ws, stream)) != DVNR_OK) return rc;
    RenderBlock& b = blocks[(size_t)i];
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = (float)m->box.lo[a];
      b.hi[a] = (float)m->box.hi[a];
      b.e[a] = (int32_t)(m->box.hi[a] - m->box.lo[a]);
    }
    b.pad = 0;
    b.grid = m->grid_ws;
  }
  std::stable_sort(blocks.begin(), blocks.end(),
                   [](const RenderBlock& a, const RenderBlock& b) { return a.lo[2] < b.lo[2]; });
  RenderBlock* dblocks = nullptr;
  DVNR_CUDA(dev_malloc_async(reinterpret_cast<void**>(&dblocks), blocks.size() * sizeof(RenderBlock), s));
  const cudaError_t e = cudaMemcpyAsync(dblocks, blocks.data(), blocks.size() * sizeof(RenderBlock),
                                        cudaMemcpyHostToDevice, s);
  rc = e == cudaSuccess ? launch_render(dblocks, n, lo, hi, *tf, w, h, spr, rgba_dev, s)
                        : cuda_status(e, "dvnr_render");
  dev_free_async(dblocks, s);
  if (rc == DVNR_OK) DVNR_CUDA(cudaStreamSynchronize(s));  // the host block table is released
  return rc;
}

static dvnr_status check_inr(const dvnr_model* models, int32_t n) {
  for (int i = 0; i < n; ++i) {
    if (models[i]->precision != models[0]->precision)
      return fail(DVNR_E_INVALID, "model %d: all models must use one precision", i);
    if (models[0]->precision == DVNR_FP16 && !mp_supported(models[i]))
      return fail(DVNR_E_UNSUPPORTED, "FP16 path needs n_levels*n_features <= 64, width 16, 32 or 64 and 1, 2, 4 or 8 features per level");
  }
  return DVNR_OK;
}

dvnr_status dvnr_render(const dvnr_model* models, int32_t n, const dvnr_tf* tf, int32_t w, int32_t h,
                        int32_t spr, float* rgba_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_render");
  g_err[0] = 0;
  dvnr_status rc = check_render(models, n, tf, w, h, spr, rgba_dev);
  if (rc != DVNR_OK) return rc;
  float lo[3], hi[3];
  union_frame(models, n, lo, hi);
  return render_grid(models, n, lo, hi, tf, w, h, spr, rgba_dev, stream);
}

dvnr_status dvnr_render_in_frame(const dvnr_model* models, int32_t n, const int64_t frame_lo[3],
                                 const int64_t frame_hi[3], const dvnr_tf* tf, int32_t w, int32_t h,
                                 int32_t spr, int32_t from_network, float* rgba_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_render_in_frame");
  g_err[0] = 0;
  dvnr_status rc = check_render(models, n, tf, w, h, spr, rgba_dev);
  if (rc != DVNR_OK) return rc;
  if (!frame_lo || !frame_hi) return fail(DVNR_E_INVALID, "NULL frame");
  float lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (frame_hi[a] <= frame_lo[a]) return fail(DVNR_E_INVALID, "frame must have hi > lo on every axis");
    lo[a] = (float)frame_lo[a];
    hi[a] = (float)frame_hi[a];
  }
  if (!from_network) return render_grid(models, n, lo, hi, tf, w, h, spr, rgba_dev, stream);
  if ((rc = check_inr(models, n)) != DVNR_OK) return rc;
  if ((rc = use_device(models[0])) != DVNR_OK) return rc;
  return render_inr(models, n, lo, hi, *tf, w, h, spr, rgba_dev, (cudaStream_t)stream);
}

dvnr_status dvnr_composite(const float* const* rgba_dev, const double* depth_host, int32_t n, int32_t w,
                           int32_t h, float* out_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_composite");
  g_err[0] = 0;
  if (n < 1 || !rgba_dev || !depth_host || !out_dev) return fail(DVNR_E_INVALID, "NULL argument or n < 1");
  if (w < 1 || h < 1) return fail(DVNR_E_INVALID, "w, h must be >= 1");
  for (int i = 0; i < n; ++i)
    if (!rgba_dev[i]) return fail(DVNR_E_INVALID, "image %d is NULL", i);
  std::vector<int> order((size_t)n);
  for (int i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return depth_host[a] < depth_host[b]; });
  return composite(rgba_dev, order.data(), n, (int64_t)w * h, out_dev, (cudaStream_t)stream);
}

dvnr_status dvnr_render_inr(const dvnr_model* models, int32_t n, const dvnr_tf* tf, int32_t w,
                            int32_t h, int32_t spr, float* rgba_dev, void* stream) {
  dvnr::ApiRange nvtx_("dvnr_render_inr");
  g_err[0] = 0;
  dvnr_status rc = check_render(models, n, tf, w, h, spr, rgba_dev);
  if (rc != DVNR_OK) return rc;
  if ((rc = check_inr(models, n)) != DVNR_OK) return rc;
  if ((rc = use_device(models[0])) != DVNR_OK) return rc;
  float lo[3], hi[3];
  union_frame(models, n, lo, hi);
  return render_inr(models, n, lo, hi, *tf, w, h, spr, rgba_dev, (cudaStream_t)stream);
}

dvnr_status dvnr_error_stats(const float* a_dev, const float* b_dev, int64_t n, double* out_host,
                             void* stream) {
  if (!out_host || n < 0 || (n > 0 && (!a_dev || !b_dev))) return fail(DVNR_E_INVALID, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* d = nullptr;
  DVNR_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d), 2 * sizeof(double), s));
  dvnr_status rc = launch_error_stats(a_dev, b_dev, n, d, s);
  if (rc == DVNR_OK) {
    cudaError_t e = cudaMemcpyAsync(out_host, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_status(e, "dvnr_error_stats");
  }
  dev_free_async(d, s);
  return rc;
}

dvnr_status dvnr_corner_indices(dvnr_model m, const uint32_t* coords_dev, int64_t n, uint32_t* idx_dev,
                                void* stream) {
  if (!m || n < 0 || (n > 0 && (!coords_dev || !idx_dev))) return fail(DVNR_E_INVALID, "bad argument");
  dvnr_status rc = use_device(m);
  if (rc != DVNR_OK) return rc;
  return launch_corner_indices(m, coords_dev, n, idx_dev, (cudaStream_t)stream);
}

}  // extern "C"
