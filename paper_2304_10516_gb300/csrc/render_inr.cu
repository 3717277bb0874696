// render_inr.cu -- direct volume rendering of DVNR models without decoding
// them to a grid (Sec. 4.3: the renderer evaluates the network at the ray
// samples, keeping the memory footprint of the compressed form).
//
// Camera, sampling and transfer function are those of render.cu: orthographic
// rays along +z, one per pixel centre, over the union of the owned boxes; spr
// samples at the centres of spr equal steps in z; a sample belongs to the
// block whose half-open box [lo - 1/2, hi - 1/2) contains it; linear RGBA
// transfer function; front-to-back compositing without early termination.
// The value at a sample is the block's network evaluated at the sample's
// position (global voxel coordinates mapped into the block's unit domain,
// clamped to it), de-normalised with the block's value range.
//
// Work unit: a group of up to 128 rays of one block (consecutive pixels of
// its footprint, row-major, so a group is mostly one image row) marched
// through all of the block's samples. Thread i owns ray i of the group and
// composites its samples front to back in registers; one tile of 128
// samples holds the group's samples at one depth, x-adjacent, which is the
// access pattern of grid decoding (neighbouring cells, neighbouring table
// entries). The result per (block, ray) is a pair (C, T): premultiplied
// colour and transmittance. Pairs compose front to back as
// (C1, T1) o (C2, T2) = (C1 + T1 C2, T1 T2), so blocks are independent and a
// second pass blends them per pixel in depth order.
//  * FP16 models: one persistent tcgen05 kernel generates the coordinates,
//    gathers the hash grid, runs the MLP on the tensor cores and composites
//    (coordinates, inference and shading fused).
//  * FP32 models: the paper's sample streaming -- a kernel writes the
//    coordinates of a chunk of rays, the FP32 decoder evaluates them, and a
//    shading kernel composites each ray.
#include <algorithm>
#include <vector>

#include "mp_common.cuh"

namespace dvnr {

namespace {

constexpr int kGroup = 128;  // rays per group (= rows of one MMA tile)

struct InrFrame {
  float lo[3], hi[3];  // union of the owned boxes (global voxel indices)
  int32_t w, h, spr;
  dvnr_tf tf;
};

// One model's share of the frame: the pixels whose ray centre falls in its
// box (px0 .. px0+npx-1, py0 .. py0+npy-1) and the samples k0 .. k0+nk-1 of
// those rays inside it. Its rays (row-major over the footprint) have
// composites ray0 .. ray0 + npx npy - 1 and form groups grp0 .. of kGroup.
struct InrBlock {
  const __half* theta16;
  const ModelState* st;
  float origin[3];  // global coordinate of stored voxel 0 (lo - ghost)
  int32_t nstore[3];
  int32_t px0, npx, py0, npy, k0, nk;
  int64_t ray0, grp0;
};

struct InrParams {
  LevelTab lv;
  int32_t D, H;
  int64_t w_off[kMaxHidden + 1];
  MpLayout lay;
  const InrBlock* blocks;
  int32_t n_blocks;
  int64_t n_grp;
  InrFrame fr;
  float4* part;  // (C.r, C.g, C.b, T) per (block, ray)
};

__host__ __device__ __forceinline__ float frame_x(const InrFrame& f, int px) {
  return (f.lo[0] - 0.5f) + ((px + 0.5f) * (f.hi[0] - f.lo[0])) / (float)f.w;
}
__host__ __device__ __forceinline__ float frame_y(const InrFrame& f, int py) {
  return (f.lo[1] - 0.5f) + ((py + 0.5f) * (f.hi[1] - f.lo[1])) / (float)f.h;
}
__host__ __device__ __forceinline__ float frame_z(const InrFrame& f, int k) {
  return (f.lo[2] - 0.5f) + ((k + 0.5f) * (f.hi[2] - f.lo[2])) / (float)f.spr;
}

// Transfer function of one value: opacity and colour (render.cu's).
__device__ __forceinline__ void apply_tf(const dvnr_tf& tf, float v, float& a, float& r, float& g,
                                         float& b) {
  const float span = tf.v_hi - tf.v_lo;
  float vn = span > 0.f ? (v - tf.v_lo) / span : 0.f;
  vn = fminf(fmaxf(vn, 0.f), 1.f);
  a = tf.alpha_max * vn;
  r = tf.c0[0] + (tf.c1[0] - tf.c0[0]) * vn;
  g = tf.c0[1] + (tf.c1[1] - tf.c0[1]) * vn;
  b = tf.c0[2] + (tf.c1[2] - tf.c0[2]) * vn;
}

// Block of group g: the last block whose grp0 <= g (blocks in grp0 order;
// blocks without rays share grp0 with their successor and are skipped).
__device__ __forceinline__ int block_of(const InrBlock* blocks, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blocks[mid].grp0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One front-to-back step of a ray's composite.
__device__ __forceinline__ void blend(float4& acc, float a, float r, float g, float b) {
  const float wgt = acc.w * a;
  acc.x += wgt * r;
  acc.y += wgt * g;
  acc.z += wgt * b;
  acc.w *= 1.f - a;
}

// FP16 models: coordinates, inference and shading in one persistent
// kernel. Each CTA walks a contiguous run of ray groups (so the network
// weights in shared memory change only at block boundaries) and marches
// every group front to back through its block, one depth per tile.
template <int W, int F>
__global__ void __launch_bounds__(kTile) k_mp_render_inr(const __grid_constant__ InrParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 8);
  volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(smem + 12);
  uint8_t* s_act = smem + p.lay.smem_act;
  const float* s_wout = reinterpret_cast<const float*>(smem + p.lay.smem_wout);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int D = p.D, H = p.H;
  const int64_t g_begin = (p.n_grp * blockIdx.x) / gridDim.x;
  const int64_t g_end = (p.n_grp * (blockIdx.x + 1)) / gridDim.x;
  if (g_begin >= g_end) return;
  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    *abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, p.lay.tmem_cols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  int b = block_of(p.blocks, p.n_blocks, g_begin);
  int cur = -1;
  InrBlock bk{};
  float vmin = 0.f, range = 0.f;

  for (int64_t grp = g_begin; grp < g_end; ++grp) {
    while (b + 1 < p.n_blocks && p.blocks[b + 1].grp0 <= grp) ++b;
    if (b != cur) {
      cur = b;
      bk = p.blocks[b];
      float inv_range;
      value_range(bk.st, vmin, inv_range);
      range = inv_range > 0.f ? ordered_to_float(bk.st->enc_max) - vmin : 0.f;
      load_weights(bk.theta16, p.w_off, D, H, W, p.lay, smem);
    }
    const int64_t ray = (grp - bk.grp0) * kGroup + tid;  // ray of this thread in the block
    const bool valid = ray < (int64_t)bk.npx * bk.npy;
    uint32_t mx = 0u, my = 0u;
    if (valid) {
      const int px = bk.px0 + (int)(ray % bk.npx), py = bk.py0 + (int)(ray / bk.npx);
      mx = dec_unit_to_fixed(frame_x(p.fr, px), bk.origin[0], bk.nstore[0]);
      my = dec_unit_to_fixed(frame_y(p.fr, py), bk.origin[1], bk.nstore[1]);
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 1.f);
    for (int kk = 0; kk < bk.nk; ++kk) {
      const uint3 m = make_uint3(mx, my, dec_unit_to_fixed(frame_z(p.fr, bk.k0 + kk), bk.origin[2],
                                                           bk.nstore[2]));
      encode_to_tile<F, DVNR_DEC_PAIR, DVNR_DEC_GROUP>(p.lv, bk.theta16, m, valid, s_act,
                                                       (uint32_t)tid);
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      float h[W];
      for (int k = 0; k < H; ++k) {
        if (tid == 0) {
          umma::fence_after_sync();
          issue_forward(tmem, smem, p.lay, k, k == 0 ? D : W, W);
          umma::commit(mbar);
        }
        umma::mbar_wait_bounded(mbar, phase, abort_flag, kWaitCycles);
        phase ^= 1u;
        __syncthreads();
        if (*abort_flag) goto teardown;
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
            *reinterpret_cast<uint4*>(s_act + tile_off(f0 + c * 8, tid)) = u;
          }
          umma::fence_proxy_async();
        } else {
#pragma unroll
          for (int j = 0; j < W; ++j) h[j] = __half2float(__float2half_rn(fmaxf(h[j], 0.f)));
        }
        umma::fence_before_sync();
        __syncthreads();
      }
      float y = 0.f;
#pragma unroll
      for (int j = 0; j < W; ++j) y += h[j] * s_wout[j];
      float a, r, g, bl;
      apply_tf(p.fr.tf, y * range + vmin, a, r, g, bl);
      blend(acc, a, r, g, bl);
    }
    if (valid) p.part[bk.ray0 + ray] = acc;
    __syncthreads();  // s_wout may be reloaded for the next block
  }
teardown:
  if (*abort_flag && tid == 0) {
    const long long t0 = clock64();
    while (!umma::mbar_try_wait(mbar, phase) && clock64() - t0 < kWaitCycles) {
    }
    if (cur >= 0) atomicAdd(const_cast<uint32_t*>(&bk.st->timeouts), 1u);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, p.lay.tmem_cols);
}

// FP32 models, step 1 of the sample streaming: fixed-point coordinates of
// the samples of rays [r0, r0 + nr) of one block, depth-major (sample k of
// ray r at (k - k0) nr + r - r0) so that step 3 reads them coalesced.
__global__ void k_inr_coords(InrBlock bk, InrFrame fr, int64_t r0, int64_t nr,
                             uint32_t* __restrict__ coords) {
  const int64_t n = nr * bk.nk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = bk.k0 + (int)(i / nr);
    const int64_t ray = r0 + i % nr;
    const int px = bk.px0 + (int)(ray % bk.npx), py = bk.py0 + (int)(ray / bk.npx);
    coords[3 * i] = dec_unit_to_fixed(frame_x(fr, px), bk.origin[0], bk.nstore[0]);
    coords[3 * i + 1] = dec_unit_to_fixed(frame_y(fr, py), bk.origin[1], bk.nstore[1]);
    coords[3 * i + 2] = dec_unit_to_fixed(frame_z(fr, k), bk.origin[2], bk.nstore[2]);
  }
}

// FP32 models, step 3: one thread per ray of [r0, r0 + nr) composites its
// decoded values front to back.
__global__ void k_inr_shade(InrBlock bk, dvnr_tf tf, int64_t r0, int64_t nr,
                            const float* __restrict__ values, float4* __restrict__ part) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 1.f);
  for (int kk = 0; kk < bk.nk; ++kk) {
    float a, cr, cg, cb;
    apply_tf(tf, values[(int64_t)kk * nr + r], a, cr, cg, cb);
    blend(acc, a, cr, cg, cb);
  }
  part[bk.ray0 + r0 + r] = acc;
}

// Blend the blocks of every pixel front to back: blocks in order of lo.z
// (disjoint boxes, so this is the depth order along every ray).
// rgba = (C, 1 - T).
__global__ void k_inr_composite(const InrBlock* __restrict__ blocks, int nb, int w, int h,
                                const float4* __restrict__ part, float* __restrict__ rgba) {
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)w * h) return;
  const int px = (int)(pix % w), py = (int)(pix / w);
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
  for (int b = 0; b < nb; ++b) {
    const InrBlock bk = blocks[b];
    const int rx = px - bk.px0, ry = py - bk.py0;
    if (rx < 0 || rx >= bk.npx || ry < 0 || ry >= bk.npy) continue;
    const float4 c = part[bk.ray0 + (int64_t)ry * bk.npx + rx];
    C0 += T * c.x;
    C1 += T * c.y;
    C2 += T * c.z;
    T *= c.w;
  }
  reinterpret_cast<float4*>(rgba)[pix] = make_float4(C0, C1, C2, 1.f - T);
}

template <int W, int F>
void launch_render_inr_wf(const InrParams& p, cudaStream_t s) {
  cudaFuncSetAttribute(k_mp_render_inr<W, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)p.lay.smem_bytes);
  const int per_sm = resident_ctas(k_mp_render_inr<W, F>, kTile, p.lay.smem_bytes, p.lay.ctas_per_sm);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(p.n_grp, (int64_t)sm_count() * per_sm));
  k_mp_render_inr<W, F><<<grid, kTile, p.lay.smem_bytes, s>>>(p);
}

// First index in [0, n) whose coordinate lies at or after `edge` (the same
// single-precision expression as the kernels), by scanning.
template <class Fn>
int first_at_or_after(int n, float edge, Fn coord) {
  int i = 0;
  while (i < n && !(coord(i) >= edge)) ++i;
  return i;
}

}  // namespace

dvnr_status render_inr(const dvnr_model* models, int n, const float* frame_lo, const float* frame_hi,
                       const dvnr_tf& tf, int w, int h, int spr, float* rgba, cudaStream_t s) {
  const bool fp16 = models[0]->precision == DVNR_FP16;
  InrFrame fr{};
  for (int a = 0; a < 3; ++a) {
    fr.lo[a] = frame_lo[a];
    fr.hi[a] = frame_hi[a];
  }
  fr.w = w;
  fr.h = h;
  fr.spr = spr;
  fr.tf = tf;
  // blocks front to back (lo.z), each with its pixel footprint and samples
  std::vector<int> order((size_t)n);
  for (int i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return models[a]->box.lo[2] < models[b]->box.lo[2]; });
  std::vector<InrBlock> blocks((size_t)n);
  int64_t n_ray = 0, n_grp = 0;
  for (int j = 0; j < n; ++j) {
    const dvnr_model m = models[order[(size_t)j]];
    InrBlock& bk = blocks[(size_t)j];
    bk = InrBlock{};
    bk.theta16 = m->theta16;
    bk.st = m->st;
    for (int a = 0; a < 3; ++a) {
      bk.origin[a] = (float)(m->box.lo[a] - m->box.ghost);
      bk.nstore[a] = (int32_t)m->dims[a];
    }
    const float xl = (float)m->box.lo[0] - 0.5f, xh = (float)m->box.hi[0] - 0.5f;
    const float yl = (float)m->box.lo[1] - 0.5f, yh = (float)m->box.hi[1] - 0.5f;
    const float zl = (float)m->box.lo[2] - 0.5f, zh = (float)m->box.hi[2] - 0.5f;
    auto fx = [&](int i) { return frame_x(fr, i); };
    auto fy = [&](int i) { return frame_y(fr, i); };
    auto fz = [&](int i) { return frame_z(fr, i); };
    bk.px0 = first_at_or_after(w, xl, fx);
    bk.npx = first_at_or_after(w, xh, fx) - bk.px0;
    bk.py0 = first_at_or_after(h, yl, fy);
    bk.npy = first_at_or_after(h, yh, fy) - bk.py0;
    bk.k0 = first_at_or_after(spr, zl, fz);
    bk.nk = first_at_or_after(spr, zh, fz) - bk.k0;
    if (bk.npx <= 0 || bk.npy <= 0 || bk.nk <= 0) bk.npx = bk.npy = bk.nk = 0;
    const int64_t rays = (int64_t)bk.npx * bk.npy;
    bk.ray0 = n_ray;
    bk.grp0 = n_grp;
    n_ray += rays;
    n_grp += (rays + kGroup - 1) / kGroup;
  }
  // FP16: one fused launch per configuration class, each over a table of
  // its blocks with groups renumbered from 0 (composites keep their global
  // ray0); the depth-ordered table for the final blend follows them
  std::vector<std::vector<int>> classes;  // indices into `blocks`
  if (fp16) {
    for (int j = 0; j < n; ++j) {
      const dvnr_model m = models[order[(size_t)j]];
      bool placed = false;
      for (auto& c : classes)
        if (same_arch(models[order[(size_t)c[0]]], m)) {
          c.push_back(j);
          placed = true;
          break;
        }
      if (!placed) classes.push_back({j});
    }
  }
  std::vector<InrBlock> table(blocks);
  std::vector<int64_t> class_grps;
  for (const auto& c : classes) {
    int64_t g = 0;
    for (int j : c) {
      InrBlock bk = blocks[(size_t)j];
      bk.grp0 = g;
      g += ((int64_t)bk.npx * bk.npy + kGroup - 1) / kGroup;
      table.push_back(bk);
    }
    class_grps.push_back(g);
  }
  InrBlock* dblocks = nullptr;
  float4* part = nullptr;
  DVNR_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dblocks), table.size() * sizeof(InrBlock), s));
  DVNR_CUDA(cudaMemcpyAsync(dblocks, table.data(), table.size() * sizeof(InrBlock),
                            cudaMemcpyHostToDevice, s));
  DVNR_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&part), (size_t)std::max<int64_t>(n_ray, 1) * sizeof(float4), s));
  dvnr_status rc = DVNR_OK;
  if (n_grp > 0 && fp16) {
    size_t first = (size_t)n;
    for (size_t ci = 0; ci < classes.size() && rc == DVNR_OK; ++ci) {
      const dvnr_model m0 = models[order[(size_t)classes[ci][0]]];
      const size_t nb = classes[ci].size();
      InrParams p{};
      if (class_grps[ci] == 0) {
        first += nb;
        continue;
      }
      if (!make_layout(m0, false, p.lay)) {
        set_error("FP16 path: configuration exceeds shared or tensor memory");
        rc = DVNR_E_UNSUPPORTED;
        break;
      }
      p.lv = m0->lv;
      p.D = m0->lv.in_dim;
      p.H = m0->mlp.n_hidden;
      for (int k = 0; k <= m0->mlp.n_hidden; ++k) p.w_off[k] = m0->w_off[k];
      p.blocks = dblocks + first;
      p.n_blocks = (int32_t)nb;
      p.n_grp = class_grps[ci];
      p.fr = fr;
      p.part = part;
      const int W = m0->mlp.width, F = m0->lv.F;
      {
        ProfScope ps("render_inr_fp16", s);
        DVNR_WF_DISPATCH(W, F, launch_render_inr_wf, p, s);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_status(e, "render_inr");
      first += nb;
    }
  } else if (n_grp > 0) {
    // sample streaming in chunks of rays, at most ~2^24 samples per chunk
    uint32_t* coords = nullptr;
    float* values = nullptr;
    int64_t cap = 0;
    for (int j = 0; j < n && rc == DVNR_OK; ++j) {
      const InrBlock& bk = blocks[(size_t)j];
      const int64_t rays = (int64_t)bk.npx * bk.npy;
      if (rays == 0) continue;
      const dvnr_model m = models[order[(size_t)j]];
      const int64_t chunk = std::max<int64_t>(1, (1LL << 24) / bk.nk);
      const int64_t need = std::min(rays, chunk) * bk.nk;
      if (need > cap) {
        if (coords) cudaFreeAsync(coords, s);
        if (values) cudaFreeAsync(values, s);
        coords = nullptr;
        values = nullptr;
        cudaError_t e1 = cudaMallocAsync(reinterpret_cast<void**>(&coords), (size_t)need * 12, s);
        cudaError_t e2 = cudaMallocAsync(reinterpret_cast<void**>(&values), (size_t)need * 4, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
          rc = cuda_status(e1 != cudaSuccess ? e1 : e2, "render_inr workspace");
          break;
        }
        cap = need;
      }
      for (int64_t r0 = 0; r0 < rays && rc == DVNR_OK; r0 += chunk) {
        const int64_t nr = std::min(chunk, rays - r0);
        const int64_t ns = nr * bk.nk;
        {
          ProfScope ps("render_inr_coords", s);
          k_inr_coords<<<(unsigned)std::min<int64_t>((ns + 255) / 256, 152 * 32), 256, 0, s>>>(
              bk, fr, r0, nr, coords);
        }
        if ((rc = fp32_decode_unit(m, coords, nullptr, ns, 0, values, s)) != DVNR_OK) break;
        {
          ProfScope ps("render_inr_shade", s);
          k_inr_shade<<<(unsigned)((nr + 127) / 128), 128, 0, s>>>(bk, tf, r0, nr, values, part);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_status(e, "render_inr");
      }
    }
    if (coords) cudaFreeAsync(coords, s);
    if (values) cudaFreeAsync(values, s);
  }
  if (rc == DVNR_OK) {
    const int64_t npix = (int64_t)w * h;
    ProfScope ps("render_inr_composite", s);
    k_inr_composite<<<(unsigned)((npix + 127) / 128), 128, 0, s>>>(dblocks, n, w, h, part, rgba);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_status(e, "render_inr");
  }
  cudaFreeAsync(part, s);
  cudaFreeAsync(dblocks, s);
  if (rc == DVNR_OK) DVNR_CUDA(cudaStreamSynchronize(s));  // the host block table is released
  return rc;
}

namespace {

// Sort-last blend of n premultiplied RGBA images, imgs[0] frontmost.
__global__ void k_composite(const float4* const* __restrict__ imgs, int n, int64_t npix,
                            float4* __restrict__ out) {
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = 0; i < n; ++i) {
    const float4 c = imgs[i][pix];
    const float t = 1.f - acc.w;
    acc.x += t * c.x;
    acc.y += t * c.y;
    acc.z += t * c.z;
    acc.w += t * c.w;
  }
  out[pix] = acc;
}

}  // namespace

dvnr_status composite(const float* const* rgba, const int* order, int n, int64_t npix, float* out,
                      cudaStream_t s) {
  std::vector<const float4*> ptrs((size_t)n);
  for (int i = 0; i < n; ++i) ptrs[(size_t)i] = reinterpret_cast<const float4*>(rgba[order[i]]);
  const float4** d = nullptr;
  DVNR_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), (size_t)n * sizeof(float4*), s));
  DVNR_CUDA(cudaMemcpyAsync(d, ptrs.data(), (size_t)n * sizeof(float4*), cudaMemcpyHostToDevice, s));
  dvnr_status rc = DVNR_OK;
  {
    ProfScope ps("composite", s);
    k_composite<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(d, n, npix, reinterpret_cast<float4*>(out));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) rc = cuda_status(e, "composite");
  cudaFreeAsync(d, s);
  if (rc == DVNR_OK) DVNR_CUDA(cudaStreamSynchronize(s));  // the host pointer table is released
  return rc;
}

}  // namespace dvnr
