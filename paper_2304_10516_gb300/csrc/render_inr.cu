// render_inr.cu -- direct volume rendering of DVNR models without decoding
// them to a grid (Sec. 4.3: the renderer evaluates the network at the ray
// samples, keeping the memory footprint of the compressed form), and the
// sort-last blend of images rendered apart.
//
// Camera, sampling and transfer function are those of render.cu: orthographic
// rays along +z, one per pixel centre, over a frame box; spr samples at the
// centres of spr equal steps in z; a sample belongs to the block whose
// half-open box [lo - 1/2, hi - 1/2) contains it; linear RGBA transfer
// function; front-to-back compositing without early termination. The value
// at a sample is the block's network evaluated at the sample's position
// (global voxel coordinates mapped into the block's unit domain, clamped to
// it), de-normalised with the block's value range.
//
// Sample streaming, block by block and in chunks of its rays: the block's
// decoder evaluates the chunk's samples straight from the ray lattice
// (FP16: the tcgen05 decode kernel computes the coordinates itself; FP32: a
// kernel writes them for the FP32 decoder), depth-major so that 128
// consecutive samples are 128 neighbouring rays at one depth (the access
// pattern of grid decoding); a shading kernel then composites every ray of
// the chunk front to back into a pair (C, T) -- premultiplied colour and
// transmittance -- per (block, ray). Pairs compose front to back as
// (C1, T1) o (C2, T2) = (C1 + T1 C2, T1 T2), so a last kernel blends the
// blocks of every pixel in depth order.
#include <algorithm>
#include <vector>

#include "dvnr_internal.cuh"
#include "mp_path.cuh"

namespace dvnr {

namespace {

// One model's share of the frame (its ray footprint and samples) and the
// index of its first (C, T) pair.
struct InrBlock {
  RayBlock rb;
  int64_t ray0;
};

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

__device__ __forceinline__ uint32_t unit_fixed(float g, float origin, int32_t n) {
  // u = (g - origin) / (n - 1), clamped to [0, 1], to the nearest 2^-24 (the
  // mapping of point decoding)
  if (n < 2) return 0u;
  float u = (g - origin) / (float)(n - 1);
  u = fminf(fmaxf(u, 0.f), 1.f);
  return (uint32_t)__float2uint_rn(u * 16777216.0f);
}

// FP32 models, step 1: fixed-point coordinates of the samples of rays
// [r0, r0 + nr) of one block, depth-major ((k - k0) nr + ray - r0).
__global__ void k_inr_coords(RayBlock rb, RayFrame fr, int64_t r0, int64_t nr,
                             uint32_t* __restrict__ coords) {
  const int64_t n = nr * rb.nk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = rb.k0 + (int)(i / nr);
    const int64_t ray = r0 + i % nr;
    const int px = rb.px0 + (int)(ray % rb.npx), py = rb.py0 + (int)(ray / rb.npx);
    coords[3 * i] = unit_fixed(frame_x(fr, px), rb.origin[0], rb.nstore[0]);
    coords[3 * i + 1] = unit_fixed(frame_y(fr, py), rb.origin[1], rb.nstore[1]);
    coords[3 * i + 2] = unit_fixed(frame_z(fr, k), rb.origin[2], rb.nstore[2]);
  }
}

// Step 3: one thread per ray of [r0, r0 + nr) composites its decoded values
// front to back into (C, T).
__global__ void k_inr_shade(int32_t nk, int64_t ray0, dvnr_tf tf, int64_t r0, int64_t nr,
                            const float* __restrict__ values, float4* __restrict__ part) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
  for (int kk = 0; kk < nk; ++kk) {
    float a, cr, cg, cb;
    apply_tf(tf, values[(int64_t)kk * nr + r], a, cr, cg, cb);
    const float wgt = T * a;
    C0 += wgt * cr;
    C1 += wgt * cg;
    C2 += wgt * cb;
    T *= 1.f - a;
  }
  part[ray0 + r0 + r] = make_float4(C0, C1, C2, T);
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
    const int rx = px - bk.rb.px0, ry = py - bk.rb.py0;
    if (rx < 0 || rx >= bk.rb.npx || ry < 0 || ry >= bk.rb.npy) continue;
    const float4 c = part[bk.ray0 + (int64_t)ry * bk.rb.npx + rx];
    C0 += T * c.x;
    C1 += T * c.y;
    C2 += T * c.z;
    T *= c.w;
  }
  reinterpret_cast<float4*>(rgba)[pix] = make_float4(C0, C1, C2, 1.f - T);
}

// First index in [0, n) whose coordinate lies at or after `edge` (the same
// single-precision expression as the kernels), by scanning.
template <class Fn>
int first_at_or_after(int n, float edge, Fn coord) {
  int i = 0;
  while (i < n && !(coord(i) >= edge)) ++i;
  return i;
}

constexpr int64_t kChunkSamples = 1LL << 24;  // samples decoded per chunk (64 MB of values)

}  // namespace

dvnr_status render_inr(const dvnr_model* models, int n, const float* frame_lo, const float* frame_hi,
                       const dvnr_tf& tf, int w, int h, int spr, float* rgba, cudaStream_t s) {
  const bool fp16 = models[0]->precision == DVNR_FP16;
  RayFrame fr{};
  for (int a = 0; a < 3; ++a) {
    fr.lo[a] = frame_lo[a];
    fr.hi[a] = frame_hi[a];
  }
  fr.w = w;
  fr.h = h;
  fr.spr = spr;
  // blocks front to back (lo.z), each with its pixel footprint and samples
  std::vector<int> order((size_t)n);
  for (int i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return models[a]->box.lo[2] < models[b]->box.lo[2]; });
  std::vector<InrBlock> blocks((size_t)n);
  int64_t n_ray = 0, max_chunk = 0;
  for (int j = 0; j < n; ++j) {
    const dvnr_model m = models[order[(size_t)j]];
    InrBlock& bk = blocks[(size_t)j];
    bk = InrBlock{};
    RayBlock& rb = bk.rb;
    for (int a = 0; a < 3; ++a) {
      rb.origin[a] = (float)(m->box.lo[a] - m->box.ghost);
      rb.nstore[a] = (int32_t)m->dims[a];
    }
    const float xl = (float)m->box.lo[0] - 0.5f, xh = (float)m->box.hi[0] - 0.5f;
    const float yl = (float)m->box.lo[1] - 0.5f, yh = (float)m->box.hi[1] - 0.5f;
    const float zl = (float)m->box.lo[2] - 0.5f, zh = (float)m->box.hi[2] - 0.5f;
    auto fx = [&](int i) { return frame_x(fr, i); };
    auto fy = [&](int i) { return frame_y(fr, i); };
    auto fz = [&](int i) { return frame_z(fr, i); };
    rb.px0 = first_at_or_after(w, xl, fx);
    rb.npx = first_at_or_after(w, xh, fx) - rb.px0;
    rb.py0 = first_at_or_after(h, yl, fy);
    rb.npy = first_at_or_after(h, yh, fy) - rb.py0;
    rb.k0 = first_at_or_after(spr, zl, fz);
    rb.nk = first_at_or_after(spr, zh, fz) - rb.k0;
    if (rb.npx <= 0 || rb.npy <= 0 || rb.nk <= 0) rb.npx = rb.npy = rb.nk = 0;
    const int64_t rays = (int64_t)rb.npx * rb.npy;
    bk.ray0 = n_ray;
    n_ray += rays;
    if (rays > 0) max_chunk = std::max(max_chunk, std::min(rays, std::max<int64_t>(1, kChunkSamples / rb.nk)) * rb.nk);
  }
  InrBlock* dblocks = nullptr;
  float4* part = nullptr;
  float* values = nullptr;
  uint32_t* coords = nullptr;
  // work memory; on a failure every buffer allocated so far is released below
  cudaError_t e0 = dev_malloc_async(reinterpret_cast<void**>(&dblocks), blocks.size() * sizeof(InrBlock), s);
  if (e0 == cudaSuccess)
    e0 = cudaMemcpyAsync(dblocks, blocks.data(), blocks.size() * sizeof(InrBlock), cudaMemcpyHostToDevice, s);
  if (e0 == cudaSuccess)
    e0 = dev_malloc_async(reinterpret_cast<void**>(&part), (size_t)std::max<int64_t>(n_ray, 1) * sizeof(float4), s);
  if (e0 == cudaSuccess && max_chunk > 0) {
    e0 = dev_malloc_async(reinterpret_cast<void**>(&values), (size_t)max_chunk * 4, s);
    if (e0 == cudaSuccess && !fp16) e0 = dev_malloc_async(reinterpret_cast<void**>(&coords), (size_t)max_chunk * 12, s);
  }
  dvnr_status rc = e0 == cudaSuccess ? DVNR_OK : cuda_status(e0, "render_inr workspace");
  for (int j = 0; j < n && rc == DVNR_OK; ++j) {
    const InrBlock& bk = blocks[(size_t)j];
    const RayBlock& rb = bk.rb;
    const int64_t rays = (int64_t)rb.npx * rb.npy;
    if (rays == 0) continue;
    const dvnr_model m = models[order[(size_t)j]];
    const int64_t chunk = std::max<int64_t>(1, kChunkSamples / rb.nk);
    for (int64_t r0 = 0; r0 < rays && rc == DVNR_OK; r0 += chunk) {
      const int64_t nr = std::min(chunk, rays - r0);
      const int64_t ns = nr * rb.nk;
      if (fp16) {
        if ((rc = mp_decode_rays(m, fr, rb, r0, nr, values, s)) != DVNR_OK) break;
      } else {
        {
          ProfScope ps("render_inr_coords", s);
          k_inr_coords<<<(unsigned)std::min<int64_t>((ns + 255) / 256, 152 * 32), 256, 0, s>>>(
              rb, fr, r0, nr, coords);
        }
        if ((rc = fp32_decode_unit(m, coords, nullptr, ns, 0, values, s)) != DVNR_OK) break;
      }
      {
        ProfScope ps("render_inr_shade", s);
        k_inr_shade<<<(unsigned)((nr + 127) / 128), 128, 0, s>>>(rb.nk, bk.ray0, tf, r0, nr, values, part);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_status(e, "render_inr");
    }
  }
  if (rc == DVNR_OK) {
    const int64_t npix = (int64_t)w * h;
    ProfScope ps("render_inr_composite", s);
    k_inr_composite<<<(unsigned)((npix + 127) / 128), 128, 0, s>>>(dblocks, n, w, h, part, rgba);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_status(e, "render_inr");
  }
  dev_free_async(coords, s);
  dev_free_async(values, s);
  dev_free_async(part, s);
  dev_free_async(dblocks, s);
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
  DVNR_CUDA(dev_malloc_async(reinterpret_cast<void**>(&d), (size_t)n * sizeof(float4*), s));
  cudaError_t e = cudaMemcpyAsync(d, ptrs.data(), (size_t)n * sizeof(float4*), cudaMemcpyHostToDevice, s);
  dvnr_status rc = DVNR_OK;
  if (e == cudaSuccess) {
    ProfScope ps("composite", s);
    k_composite<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(d, n, npix, reinterpret_cast<float4*>(out));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) rc = cuda_status(e, "composite");
  dev_free_async(d, s);
  if (rc == DVNR_OK) DVNR_CUDA(cudaStreamSynchronize(s));  // the host pointer table is released
  return rc;
}

}  // namespace dvnr
