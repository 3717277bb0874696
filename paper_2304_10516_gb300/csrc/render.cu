// render.cu -- direct volume rendering of decoded DVNR blocks (Sec. 4.3 of
// the paper renders the distributed representation with sort-last
// compositing; here all blocks are resident on one GPU, so compositing is an
// in-kernel front-to-back blend in block order along the view axis).
//
// Reading (the paper gives no camera or transfer function): orthographic
// rays along +z, one per pixel centre, over the union of the owned boxes;
// spr samples at the centres of spr equal steps in z; trilinear on the
// decoded grid of the block owning the sample, clamped at that block's
// edge; linear RGBA transfer function; no early ray termination.
#include "dvnr_internal.cuh"

namespace dvnr {

namespace {

struct Frame {
  float lo[3], hi[3];
};

__global__ void __launch_bounds__(128)
    k_render(const RenderBlock* __restrict__ blocks, int nb, Frame fr, dvnr_tf tf, int w, int h,
             int spr, float* __restrict__ rgba) {
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= (int64_t)w * h) return;
  const int px = (int)(pix % w), py = (int)(pix / w);
  const float X = (fr.lo[0] - 0.5f) + ((px + 0.5f) * (fr.hi[0] - fr.lo[0])) / (float)w;
  const float Y = (fr.lo[1] - 0.5f) + ((py + 0.5f) * (fr.hi[1] - fr.lo[1])) / (float)h;
  const float dz = fr.hi[2] - fr.lo[2];
  const float span = tf.v_hi - tf.v_lo;
  float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
  for (int b = 0; b < nb; ++b) {  // blocks sorted by lo.z: front to back
    const RenderBlock blk = blocks[b];
    if (!(X >= blk.lo[0] - 0.5f && X < blk.hi[0] - 0.5f && Y >= blk.lo[1] - 0.5f &&
          Y < blk.hi[1] - 0.5f))
      continue;
    const int ex = blk.e[0], ey = blk.e[1], ez = blk.e[2];
    float qx = fminf(fmaxf(X - blk.lo[0], 0.f), (float)(ex - 1));
    float qy = fminf(fmaxf(Y - blk.lo[1], 0.f), (float)(ey - 1));
    int bx = min((int)floorf(qx), max(ex - 2, 0));
    int by = min((int)floorf(qy), max(ey - 2, 0));
    const float fx = ex > 1 ? qx - (float)bx : 0.f;
    const float fy = ey > 1 ? qy - (float)by : 0.f;
    const int sx = ex > 1 ? 1 : 0;
    const size_t sy = ey > 1 ? (size_t)ex : 0;
    const size_t szs = ez > 1 ? (size_t)ex * ey : 0;
    const float* g = blk.grid + (size_t)by * ex + bx;
    const float zlo = blk.lo[2] - 0.5f, zhi = blk.hi[2] - 0.5f;
    for (int k = 0; k < spr; ++k) {
      const float Z = (fr.lo[2] - 0.5f) + ((k + 0.5f) * dz) / (float)spr;
      if (!(Z >= zlo && Z < zhi)) continue;
      const float qz = fminf(fmaxf(Z - blk.lo[2], 0.f), (float)(ez - 1));
      const int bz = min((int)floorf(qz), max(ez - 2, 0));
      const float fz = ez > 1 ? qz - (float)bz : 0.f;
      const float* p = g + (size_t)bz * ex * ey;
      const float v00 = (1.f - fx) * __ldg(p) + fx * __ldg(p + sx);
      const float v10 = (1.f - fx) * __ldg(p + sy) + fx * __ldg(p + sy + sx);
      const float v01 = (1.f - fx) * __ldg(p + szs) + fx * __ldg(p + szs + sx);
      const float v11 = (1.f - fx) * __ldg(p + szs + sy) + fx * __ldg(p + szs + sy + sx);
      const float v = (1.f - fz) * ((1.f - fy) * v00 + fy * v10) + fz * ((1.f - fy) * v01 + fy * v11);
      float vn = span > 0.f ? (v - tf.v_lo) / span : 0.f;
      vn = fminf(fmaxf(vn, 0.f), 1.f);
      const float alpha = tf.alpha_max * vn;
      const float t = (1.f - A) * alpha;
      C0 += t * (tf.c0[0] + (tf.c1[0] - tf.c0[0]) * vn);
      C1 += t * (tf.c0[1] + (tf.c1[1] - tf.c0[1]) * vn);
      C2 += t * (tf.c0[2] + (tf.c1[2] - tf.c0[2]) * vn);
      A += t;
    }
  }
  reinterpret_cast<float4*>(rgba)[pix] = make_float4(C0, C1, C2, A);
}

}  // namespace

dvnr_status launch_render(const RenderBlock* blocks_dev, int n_blocks, const float lo[3],
                          const float hi[3], const dvnr_tf& tf, int w, int h, int spr,
                          float* rgba, cudaStream_t s) {
  Frame fr;
  for (int a = 0; a < 3; ++a) {
    fr.lo[a] = lo[a];
    fr.hi[a] = hi[a];
  }
  const int64_t n = (int64_t)w * h;
  {
    ProfScope ps_("render", s);
    k_render<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blocks_dev, n_blocks, fr, tf, w, h, spr,
                                                       rgba);
  }
  DVNR_CUDA(cudaGetLastError());
  return DVNR_OK;
}

}  // namespace dvnr
