// probe.cu -- measurement of the training step's memory-request pattern
// alone (dvnr_probe_requests). The FP16 training kernel is bound by the rate
// at which the SMs get scattered 4- and 8-byte table entries and 16-byte
// gradient reductions through L1 and L2, not by DRAM bandwidth or the tensor
// cores. This kernel issues exactly the requests of one training step of a
// model -- the same Philox samples, volume corners, staged corner gathers of
// the FP16 tables and vector reductions into the FP32 gradients, tile by tile
// over a persistent grid -- with no MLP, at a chosen number of resident CTAs
// per SM, so that the fastest such launch is the ceiling of that request
// pattern on this GPU.
#include <algorithm>

#include "mp_common.cuh"

namespace dvnr {

namespace {

struct ProbeParams {
  LevelTab lv;
  const __half* theta16;
  float* grad;  // scratch gradient (never the model's)
  const float* vol;
  int32_t nx, ny, nz;
  SampleParams sp;
  uint32_t iter;
  int32_t batch;
  int64_t total_tiles;
  int32_t stage_levels;  // levels staged per gather round
  int32_t mode;          // bit 0: gathers, bit 1: reductions, bit 2: volume reads
  float* sink;           // keeps the gathered values alive (one float per CTA)
};

constexpr uint32_t kProbeActBytes = 4u * 16u * 128u * 2u;  // encoding tile of up to 64 features

__global__ void __launch_bounds__(kTile) k_probe_requests(const __grid_constant__ ProbeParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* s_act = smem;
  uint8_t* s_stage = smem + kProbeActBytes;
  const int tid = threadIdx.x;
  const int64_t g0 = (p.total_tiles * blockIdx.x) / gridDim.x;
  const int64_t g1 = (p.total_tiles * (blockIdx.x + 1)) / gridDim.x;
  float keep = 0.f;
  const int D = p.lv.in_dim;
  for (int64_t g = g0; g < g1; ++g) {
    const int i = (int)g * kTile + tid;
    const bool valid = i < p.batch;
    const uint3 mc = valid ? draw_sample(p.sp, (uint32_t)i, p.iter) : make_uint3(0u, 0u, 0u);
    if ((p.mode & 4) && valid) keep += vol_interp(vol_fetch(p.vol, p.nx, p.ny, p.nz, mc));
    if (p.mode & 1) {
      encode_to_tile_staged(p.lv, p.theta16, mc, valid, s_act, (uint32_t)tid, s_stage, p.stage_levels,
                            s_stage, 0);
      const __half* row = reinterpret_cast<const __half*>(s_act + tile_off(0, (uint32_t)tid));
      keep += __half2float(row[0]);
    }
    if ((p.mode & 2) && valid) {
      float d[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) d[j] = 1e-6f;
      for (int c = 0; c < D; c += 16) {
        if (c + 16 <= D)
          scatter_chunk<2, false>(p.lv, p.grad, mc, d, c);
        else
          scatter_chunk<2, true>(p.lv, p.grad, mc, d, c);
      }
    }
  }
  if (keep == 123456.f) p.sink[blockIdx.x] = keep;  // never true in practice; keeps the loads
}

}  // namespace

}  // namespace dvnr

extern "C" dvnr_status dvnr_probe_requests(dvnr_model m, const float* vol_dev, int32_t batch,
                                           int32_t ctas_per_sm, int32_t mode, int32_t iters,
                                           double* ms_out) {
  using namespace dvnr;
  if (!m || !ms_out || batch < 1 || ctas_per_sm < 1 || ctas_per_sm > 16 || iters < 1 || mode < 1 ||
      mode > 7 || ((mode & 4) && !vol_dev)) {
    set_error("bad argument");
    return DVNR_E_INVALID;
  }
  if (m->frozen) {
    set_error("the model is frozen");
    return DVNR_E_STATE;
  }
  if (m->lv.F != 2 || m->lv.in_dim > 64) {
    set_error("the probe covers two features per level and encodings of at most 64 values");
    return DVNR_E_UNSUPPORTED;
  }
  int dev = 0, smem_sm = 0;
  DVNR_CUDA(cudaGetDevice(&dev));
  DVNR_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  // dynamic shared memory sized so that at most ctas_per_sm CTAs fit per SM;
  // what is beyond the encoding tile stages gathers (4 KB per level)
  const size_t per_cta = (size_t)smem_sm / (size_t)ctas_per_sm - 1024;
  const size_t smem = std::min<size_t>(per_cta, 227 * 1024) / 1024 * 1024;
  const int stage_levels = (int)std::min<size_t>(16, (smem - kProbeActBytes) / kStageLevelBytes);
  if (smem < kProbeActBytes + kStageLevelBytes || stage_levels < 1) {
    set_error("too many CTAs per SM for the probe's shared memory");
    return DVNR_E_UNSUPPORTED;
  }
  cudaFuncSetAttribute(k_probe_requests, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_probe_requests, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  const int per_sm = resident_ctas(k_probe_requests, kTile, smem, ctas_per_sm);
  ProbeParams p{};
  p.lv = m->lv;
  p.theta16 = m->theta16;
  p.vol = vol_dev;
  p.nx = (int32_t)m->dims[0];
  p.ny = (int32_t)m->dims[1];
  p.nz = (int32_t)m->dims[2];
  p.sp.key = make_uint2(7u, 0u);
  p.sp.model = 0;
  p.sp.n_bnd = 0;
  p.sp.qtab = m->qtab;
  p.batch = batch;
  p.total_tiles = (batch + kTile - 1) / kTile;
  p.stage_levels = stage_levels;
  p.mode = mode;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(p.total_tiles, (int64_t)sm_count() * per_sm));
  cudaStream_t s = 0;
  float* scratch = nullptr;
  DVNR_CUDA(dev_malloc(reinterpret_cast<void**>(&scratch), ((size_t)m->n_store + (size_t)grid) * sizeof(float)));
  p.grad = scratch;
  p.sink = scratch + m->n_store;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemset(scratch, 0, ((size_t)m->n_store + (size_t)grid) * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // one untimed launch, then `iters` timed ones, each with its own samples
  for (int it = 0; it <= iters && e == cudaSuccess; ++it) {
    if (it == 1) e = cudaEventRecord(e0, s);
    p.iter = (uint32_t)it;
    {
      ProfScope ps("probe_requests", s);
      k_probe_requests<<<grid, kTile, smem, s>>>(p);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(scratch);
  if (e != cudaSuccess) return cuda_status(e, "dvnr_probe_requests");
  ms_out[0] = (double)ms / iters;
  ms_out[1] = (double)per_sm;
  return DVNR_OK;
}
