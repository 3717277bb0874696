// fp32_path.cu -- the plain FP32 SIMT training path of libdvnr (one model at
// a time, separate kernels per stage, no tensor cores). It is the reference
// GPU path that the FP16 tensor-core path is compared with ("equal PSNR vs
// plain FP32 path").
//
// Stages per step (Sec. 3.2): sample + target + encode -> per-layer GEMMs ->
// output + L1/L2 loss -> per-layer backward GEMMs and weight gradients ->
// dL/d(encoding) -> scatter into the table gradients. Adam is in util.cu.
#include <algorithm>

#include "dvnr_internal.cuh"

namespace dvnr {

namespace {

// ------------------------------------------------------------- encoding ----
template <int F>
struct FVec;
template <>
struct FVec<1> {
  static __device__ __forceinline__ void load(const float* p, float* v) { v[0] = __ldg(p); }
};
template <>
struct FVec<2> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = a.x;
    v[1] = a.y;
  }
};
template <>
struct FVec<4> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct FVec<8> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    FVec<4>::load(p, v);
    FVec<4>::load(p + 4, v + 4);
  }
};

// Hash-grid encoding of one coordinate in FP32 (Sec. 3; Mueller et al.):
// per level 8 corners, trilinear weights, F features, level-major output.
template <int F>
__device__ void encode_fp32(const LevelTab& lv, const float* __restrict__ theta, uint3 m,
                            float* __restrict__ out) {
  for (int l = 0; l < lv.L; ++l) {
    uint32_t bx, by, bz;
    float fx, fy, fz;
    lattice(m.x, lv.N[l], bx, fx);
    lattice(m.y, lv.N[l], by, fy);
    lattice(m.z, lv.N[l], bz, fz);
    float acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.f;
    const float* tab = theta + lv.off[l];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
      const float w = (cx ? fx : 1.f - fx) * (cy ? fy : 1.f - fy) * (cz ? fz : 1.f - fz);
      const uint32_t idx = corner_index(lv, l, bx + cx, by + cy, bz + cz);
      float v[F];
      FVec<F>::load(tab + (size_t)idx * F, v);
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] += w * v[f];
    }
#pragma unroll
    for (int f = 0; f < F; ++f) out[l * F + f] = acc[f];
  }
}

template <int F>
__global__ void k_sample_encode(LevelTab lv, const float* __restrict__ theta,
                                const float* __restrict__ vol, int nx, int ny, int nz,
                                SampleParams sp, const ModelState* __restrict__ st, int32_t batch,
                                int use_iter, uint32_t iter_arg, float* __restrict__ x0,
                                float* __restrict__ tgt, uint32_t* __restrict__ coords,
                                int gated, const uint32_t* __restrict__ ext_coords) {
  if (gated && !model_active(st)) return;  // the model's call is over (budget or early stop)
  const uint32_t iter = use_iter ? iter_arg : st->iter;
  float vmin, inv_range;
  value_range(st, vmin, inv_range);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
    if (ext_coords) {  // given points: no sampling, no target
      const uint3 m = make_uint3(ext_coords[3 * i], ext_coords[3 * i + 1], ext_coords[3 * i + 2]);
      encode_fp32<F>(lv, theta, m, x0 + (size_t)i * lv.in_dim);
      continue;
    }
    const uint3 m = draw_sample(sp, (uint32_t)i, iter);
    coords[3 * i] = m.x;
    coords[3 * i + 1] = m.y;
    coords[3 * i + 2] = m.z;
    tgt[i] = (volume_trilinear(vol, nx, ny, nz, m) - vmin) * inv_range;
    encode_fp32<F>(lv, theta, m, x0 + (size_t)i * lv.in_dim);
  }
}

// ----------------------------------------------------------------- GEMM ----
// C[M x N] = opA(M x K) opB(K x N), 64 x 64 tile per block of 256 threads,
// 4 x 4 outputs per thread, K staged 16 at a time through shared memory.
//   opA(m,k) = TA ? A[k lda + m] : A[m lda + k]
//   opB(k,n) = TB ? B[n ldb + k] : B[k ldb + n]
// EPI 0: store; 1: store ReLU; 2: store times [aux > 0] (ReLU derivative);
// 3: atomic add (split-K over blockIdx.z in chunks of kchunk).
enum { EPI_STORE = 0, EPI_RELU = 1, EPI_MASK = 2, EPI_ATOMIC = 3 };

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256)
    k_sgemm64(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
              float* __restrict__ C, int ldc, const float* __restrict__ aux, int M, int N, int K,
              int kchunk, const ModelState* __restrict__ gate) {
  if (gate && !model_active(gate)) return;
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int mm, kk;
      if (TA) { mm = e & 63; kk = e >> 6; } else { kk = e & 15; mm = e >> 4; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int nn, kk;
      if (TB) { kk = e & 15; nn = e >> 4; } else { nn = e & 63; kk = e >> 6; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      const float v = acc[i][j];
      float* c = C + (size_t)m * ldc + n;
      if (EPI == EPI_STORE) *c = v;
      if (EPI == EPI_RELU) *c = v > 0.f ? v : 0.f;
      if (EPI == EPI_MASK) *c = aux[(size_t)m * ldc + n] > 0.f ? v : 0.f;
      if (EPI == EPI_ATOMIC) atomicAdd(c, v);
    }
  }
}

template <bool TA, bool TB, int EPI>
dvnr_status gemm(const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                 const float* aux, int M, int N, int K, int splits, cudaStream_t s,
                 const ModelState* gate = nullptr) {
  const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((M + 63) / 64, (N + 63) / 64, std::max(splits, 1));
  {
    ProfScope ps_("fp32_gemm", s);
    k_sgemm64<TA, TB, EPI><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, aux, M, N, K, kchunk, gate);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

// ------------------------------------------------------- output and loss ---
// y = w_out . h_H, loss L1 (sign(y - t)/B, sign(0) = 0) or L2 (2 (y - t)/B)
// (Sec. 3.3: unweighted L1 over the mixed batch), dW_out += dy h_H,
// dZ_H = dy w_out [h_H > 0]. A non-finite output flags the step.
__global__ void __launch_bounds__(128)
    k_out_loss(const float* __restrict__ hH, const float* __restrict__ wout, int W,
               const float* __restrict__ tgt, int32_t batch, int32_t loss, float inv_B,
               float* __restrict__ dzH, float* __restrict__ gwout, ModelState* st,
               float* __restrict__ y_out, int gated, const float* __restrict__ ext_dy) {
  if (gated && !model_active(st)) return;
  __shared__ float s_g[256];
  __shared__ float s_w[256];
  for (int j = threadIdx.x; j < W; j += blockDim.x) {
    s_g[j] = 0.f;
    s_w[j] = wout[j];
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < batch;
  float dy = 0.f, lval = 0.f;
  const float* h = hH + (size_t)(valid ? i : 0) * W;
  if (valid) {
    float y = 0.f;
    for (int j = 0; j < W; ++j) y += s_w[j] * h[j];
    const float d = ext_dy ? 0.f : y - tgt[i];
    if (ext_dy) {  // the upstream gradient of given points
      dy = ext_dy[i];
    } else if (loss == DVNR_LOSS_L1) {
      lval = fabsf(d);
      dy = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv_B;
    } else {
      lval = d * d;
      dy = 2.f * d * inv_B;
    }
    if (!isfinite(y)) atomicOr(&st->overflow, 1u);
    if (y_out) y_out[i] = y;
    float* dz = dzH + (size_t)i * W;
    for (int j = 0; j < W; ++j) dz[j] = h[j] > 0.f ? dy * s_w[j] : 0.f;
  }
  for (int j = 0; j < W; ++j) {
    float g = valid ? dy * h[j] : 0.f;
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_g[j], g);
  }
  for (int o = 16; o > 0; o >>= 1) lval += __shfl_xor_sync(0xffffffffu, lval, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&st->loss_sum, lval);
  __syncthreads();
  for (int j = threadIdx.x; j < W; j += blockDim.x) atomicAdd(gwout + j, s_g[j]);
}

// ------------------------------------------------- encoding backward -------
// Table gradient += trilinear weight x dL/d(feature) for the 8 corners of
// every level (the scatter-add of the encoding's backward pass).
template <int F>
__global__ void k_scatter(LevelTab lv, const uint32_t* __restrict__ coords,
                          const float* __restrict__ dx0, int32_t batch, float* __restrict__ grad,
                          ModelState* st, float* __restrict__ dx0_out, int gated) {
  if (gated && !model_active(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
    const uint3 m = make_uint3(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]);
    const float* d = dx0 + (size_t)i * lv.in_dim;
    bool bad = false;
    for (int l = 0; l < lv.L; ++l) {
      uint32_t bx, by, bz;
      float fx, fy, fz;
      lattice(m.x, lv.N[l], bx, fx);
      lattice(m.y, lv.N[l], by, fy);
      lattice(m.z, lv.N[l], bz, fz);
      float g[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        g[f] = d[l * F + f];
        bad |= !isfinite(g[f]);
        if (dx0_out) dx0_out[(size_t)i * lv.in_dim + l * F + f] = g[f];
      }
      float* tab = grad + lv.off[l];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
        const float w = (cx ? fx : 1.f - fx) * (cy ? fy : 1.f - fy) * (cz ? fz : 1.f - fz);
        const uint32_t idx = corner_index(lv, l, bx + cx, by + cy, bz + cz);
#pragma unroll
        for (int f = 0; f < F; ++f) atomicAdd(tab + (size_t)idx * F + f, w * g[f]);
      }
    }
    if (bad) atomicOr(&st->overflow, 1u);
  }
}

// ----------------------------------------------------------- decoding ------
// Plain FP32 inference in chunks: encode kernel -> per-layer GEMMs -> output
// kernel; out = y (vmax - vmin) + vmin (Sec. 4.1 keeps the value range).
// Coordinates come from explicit fixed-point triples, from the owned voxels
// of the box (decoding back to the grid, Sec. 3) or from global voxel
// coordinates mapped into the unit domain.
struct CoordSource {
  const uint32_t* coords;  // explicit fixed-point coordinates (or NULL)
  const float* xyz;        // global voxel coordinates (or NULL)
  int grid_mode;
  int64_t e[3];            // owned voxels per axis
  int64_t nstore[3];       // stored voxels per axis
  int32_t ghost;
  float origin[3];         // global index of stored voxel 0
};

__device__ __forceinline__ uint32_t unit_to_fixed(float g, float origin, int64_t n) {
  // u = (g - origin) / (n - 1), clamped to [0, 1], to the nearest 2^-24
  if (n < 2) return 0u;
  float u = (g - origin) / (float)(n - 1);
  u = fminf(fmaxf(u, 0.f), 1.f);
  return (uint32_t)__float2uint_rn(u * 16777216.0f);
}

__device__ __forceinline__ uint32_t grid_fixed(int64_t j, int64_t n) {
  if (n < 2) return 0u;
  return (uint32_t)((2 * j * (int64_t)kFixOne + (n - 1)) / (2 * (n - 1)));
}

__device__ __forceinline__ uint3 source_coord(const CoordSource& c, int64_t i) {
  if (c.coords) return make_uint3(c.coords[3 * i], c.coords[3 * i + 1], c.coords[3 * i + 2]);
  if (c.grid_mode) {
    const int64_t x = i % c.e[0], y = (i / c.e[0]) % c.e[1], z = i / (c.e[0] * c.e[1]);
    return make_uint3(grid_fixed(x + c.ghost, c.nstore[0]), grid_fixed(y + c.ghost, c.nstore[1]),
                      grid_fixed(z + c.ghost, c.nstore[2]));
  }
  return make_uint3(unit_to_fixed(c.xyz[3 * i], c.origin[0], c.nstore[0]),
                    unit_to_fixed(c.xyz[3 * i + 1], c.origin[1], c.nstore[1]),
                    unit_to_fixed(c.xyz[3 * i + 2], c.origin[2], c.nstore[2]));
}

template <int F>
__global__ void k_decode_encode(LevelTab lv, const float* __restrict__ theta, CoordSource c,
                                int64_t first, int64_t count, float* __restrict__ x0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    encode_fp32<F>(lv, theta, source_coord(c, first + i), x0 + i * lv.in_dim);
}

__global__ void k_decode_out(const float* __restrict__ hH, const float* __restrict__ wout, int W,
                             int64_t count, const ModelState* __restrict__ st,
                             float* __restrict__ out, int raw) {
  float vmin, inv_range;
  value_range(st, vmin, inv_range);
  const float range = inv_range > 0.f ? ordered_to_float(st->enc_max) - vmin : 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* h = hH + i * W;
    float y = 0.f;
    for (int j = 0; j < W; ++j) y += __ldg(wout + j) * h[j];
    out[i] = raw ? y : y * range + vmin;
  }
}

}  // namespace

dvnr_status fp32_ensure_workspace(dvnr_model m, int64_t batch) {
  Fp32Workspace& ws = m->ws;
  if (ws.batch >= batch && ws.base) return DVNR_OK;
  if (ws.base) {
    dev_free(ws.base);
    ws = Fp32Workspace{};
  }
  const int64_t D = m->lv.in_dim, W = m->mlp.width, H = m->mlp.n_hidden;
  auto al = [](int64_t bytes) { return (bytes + 255) / 256 * 256; };
  const int64_t b_x0 = al(batch * D * 4), b_act = al(H * batch * W * 4), b_dz = al(2 * batch * W * 4),
                b_dx0 = al(batch * D * 4), b_tgt = al(batch * 4), b_c = al(batch * 12);
  void* base = nullptr;
  cudaError_t e = dev_malloc(reinterpret_cast<void**>(&base), b_x0 + b_act + b_dz + b_dx0 + b_tgt + b_c);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("FP32 workspace allocation failed (%s)", cudaGetErrorString(e));
    return DVNR_E_OOM;
  }
  char* p = static_cast<char*>(base);
  ws.base = base;
  ws.batch = batch;
  ws.x0 = reinterpret_cast<float*>(p); p += b_x0;
  ws.act = reinterpret_cast<float*>(p); p += b_act;
  ws.dz = reinterpret_cast<float*>(p); p += b_dz;
  ws.dx0 = reinterpret_cast<float*>(p); p += b_dx0;
  ws.tgt = reinterpret_cast<float*>(p); p += b_tgt;
  ws.coords = reinterpret_cast<uint32_t*>(p);
  return DVNR_OK;
}

dvnr_status fp32_forward_backward(const Fp32StepArgs& a, cudaStream_t s) {
  dvnr_model m = a.m;
  dvnr_status rc = fp32_ensure_workspace(m, a.batch);
  if (rc != DVNR_OK) return rc;
  Fp32Workspace& ws = m->ws;
  const int B = a.batch, D = m->lv.in_dim, W = m->mlp.width, H = m->mlp.n_hidden;
  const int nx = (int)m->dims[0], ny = (int)m->dims[1], nz = (int)m->dims[2];
  const int enc_blocks = std::min((B + 127) / 128, 152 * 16);
  // the scatter reads the points back: drawn ones from coords, given ones in place
  uint32_t* coords = a.coords_out ? a.coords_out : ws.coords;
  const uint32_t* scatter_coords = a.ext_coords ? a.ext_coords : coords;
  const ModelState* gate = a.gated ? m->st : nullptr;
  {
  ProfScope ps_("fp32_sample_encode", s);
  switch (m->lv.F) {
#define DVNR_SE(F)                                                                               \
  case F:                                                                                        \
    k_sample_encode<F><<<enc_blocks, 128, 0, s>>>(m->lv, m->theta, a.vol, nx, ny, nz, a.sp,     \
                                                  m->st, B, a.explicit_iter ? 1 : 0, a.iter,    \
                                                  ws.x0, ws.tgt, coords, a.gated ? 1 : 0,       \
                                                  a.ext_coords);                                \
    break;
    DVNR_SE(1) DVNR_SE(2) DVNR_SE(4) DVNR_SE(8)
#undef DVNR_SE
    default:
      return DVNR_E_UNSUPPORTED;
  }
  }
  DVNR_CUDA(cudaGetLastError());
  if (a.tgt_out && !a.ext_coords)
    DVNR_CUDA(cudaMemcpyAsync(a.tgt_out, ws.tgt, (size_t)B * 4, cudaMemcpyDeviceToDevice, s));
  // forward: H_{k+1} = ReLU(H_k W_k^T)
  const float* in = ws.x0;
  int in_dim = D;
  for (int k = 0; k < H; ++k) {
    float* outp = ws.act + (size_t)k * B * W;
    rc = gemm<false, true, EPI_RELU>(in, in_dim, m->theta + m->w_off[k], in_dim, outp, W, nullptr,
                                     B, W, in_dim, 1, s, gate);
    if (rc != DVNR_OK) return rc;
    in = outp;
    in_dim = W;
  }
  // output and loss
  float* dz = ws.dz;
  float* dz_other = ws.dz + (size_t)B * W;
  const float* hH = ws.act + (size_t)(H - 1) * B * W;
  {
  ProfScope ps_("fp32_out_loss", s);
  k_out_loss<<<(B + 127) / 128, 128, 0, s>>>(hH, m->theta + m->w_off[H], W, ws.tgt, B, a.loss,
                                             1.0f / (float)B, dz, m->grad + m->w_off[H], m->st,
                                             a.y_out, a.gated ? 1 : 0, a.ext_dy);
  }
  DVNR_CUDA(cudaGetLastError());
  const int splits = std::max(1, std::min(1024, B / 1024));
  // backward through the hidden layers: dZ_k (B x W) -> dW_{k-1}, dZ_{k-1}
  for (int k = H; k >= 1; --k) {
    const float* hprev = (k == 1) ? ws.x0 : ws.act + (size_t)(k - 2) * B * W;
    const int nin = (k == 1) ? D : W;
    float* gW = m->grad + m->w_off[k - 1];
    const float* Wk = m->theta + m->w_off[k - 1];
    rc = gemm<true, false, EPI_ATOMIC>(dz, W, hprev, nin, gW, nin, nullptr, W, nin, B, splits, s, gate);
    if (rc != DVNR_OK) return rc;
    if (k > 1) {
      rc = gemm<false, false, EPI_MASK>(dz, W, Wk, nin, dz_other, nin, hprev, B, nin, W, 1, s, gate);
      if (rc != DVNR_OK) return rc;
      std::swap(dz, dz_other);
    } else {
      rc = gemm<false, false, EPI_STORE>(dz, W, Wk, nin, ws.dx0, nin, nullptr, B, nin, W, 1, s, gate);
      if (rc != DVNR_OK) return rc;
    }
  }
  {
  ProfScope ps_("fp32_scatter", s);
  switch (m->lv.F) {
#define DVNR_SC(F)                                                                               \
  case F:                                                                                        \
    k_scatter<F><<<enc_blocks, 128, 0, s>>>(m->lv, scatter_coords, ws.dx0, B, m->grad, m->st,  \
                                            a.dx0_out, a.gated ? 1 : 0);                         \
    break;
    DVNR_SC(1) DVNR_SC(2) DVNR_SC(4) DVNR_SC(8)
#undef DVNR_SC
  }
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

dvnr_status fp32_decode_unit(dvnr_model m, const uint32_t* coords, const float* xyz, int64_t n,
                             int grid_mode, float* out, cudaStream_t s, bool raw) {
  if (n <= 0) return DVNR_OK;
  const int D = m->lv.in_dim, W = m->mlp.width, H = m->mlp.n_hidden;
  const int64_t chunk = std::min<int64_t>(n, 1 << 19);
  dvnr_status rc = fp32_ensure_workspace(m, chunk);
  if (rc != DVNR_OK) return rc;
  Fp32Workspace& ws = m->ws;
  CoordSource c{};
  c.coords = coords;
  c.xyz = xyz;
  c.grid_mode = grid_mode;
  for (int i = 0; i < 3; ++i) {
    c.e[i] = m->box.hi[i] - m->box.lo[i];
    c.nstore[i] = m->dims[i];
    c.origin[i] = (float)(m->box.lo[i] - m->box.ghost);
  }
  c.ghost = m->box.ghost;
  for (int64_t first = 0; first < n; first += chunk) {
    const int64_t cnt = std::min(chunk, n - first);
    const int blocks = (int)std::min<int64_t>((cnt + 127) / 128, 152 * 16);
    {
    ProfScope ps_("fp32_decode_encode", s);
    switch (m->lv.F) {
#define DVNR_DE(F)                                                                          \
  case F:                                                                                   \
    k_decode_encode<F><<<blocks, 128, 0, s>>>(m->lv, m->theta, c, first, cnt, ws.x0);      \
    break;
      DVNR_DE(1) DVNR_DE(2) DVNR_DE(4) DVNR_DE(8)
#undef DVNR_DE
      default:
        return DVNR_E_UNSUPPORTED;
    }
    }
    DVNR_CUDA(cudaGetLastError());
    const float* in = ws.x0;
    int in_dim = D;
    for (int k = 0; k < H; ++k) {
      float* outp = ws.dz + (size_t)(k & 1) * chunk * W;
      rc = gemm<false, true, EPI_RELU>(in, in_dim, m->theta + m->w_off[k], in_dim, outp, W, nullptr,
                                       (int)cnt, W, in_dim, 1, s);
      if (rc != DVNR_OK) return rc;
      in = outp;
      in_dim = W;
    }
    {
      ProfScope ps_("fp32_decode_out", s);
      k_decode_out<<<blocks, 128, 0, s>>>(in, m->theta + m->w_off[H], W, cnt, m->st, out + first,
                                          raw ? 1 : 0);
    }
    DVNR_CUDA(cudaGetLastError());
  }
  return DVNR_OK;
}

}  // namespace dvnr
