// mp_path.cuh -- the FP16 tensor-core (tcgen05) path of libdvnr: grouped
// persistent training kernel over many models and forward-only decoding.
#pragma once

#include "dvnr_internal.cuh"

namespace dvnr {

struct MpStepDebug {
  float* y;
  float* dx0;
  float* target;
  uint32_t* coords;
};

// True when the model's configuration is one the FP16 kernels are built for.
bool mp_supported(const dvnr_model m);
// Free the FP16-path resources of a model (graphs, descriptor tables).
void mp_release(dvnr_model m);
// `steps` grouped steps of the n models (schedule, fused kernel, reduction,
// Adam per step); a model leaves the steps once model_active is false.
// `uniform`: every model's budget equals `steps` (with no stop rule the
// schedule kernel is then skipped). All n models share one configuration;
// model i draws its samples with RNG slot slots[i].
dvnr_status mp_train(dvnr_model* models, int n, const float* const* vols, const uint32_t* slots,
                     const dvnr_train_cfg* cfg, const AdamHyper& h, int64_t steps, bool uniform,
                     cudaStream_t s);
// One forward/backward of model slot 0 at iteration `iter` and loss scale S,
// gradients left (scaled by S) in m->grad.
dvnr_status mp_train_grad(dvnr_model m, const float* vol, const dvnr_train_cfg* cfg, uint32_t iter,
                          float S, const MpStepDebug& dbg, cudaStream_t s);
// FP16 inference: xyz points (grid_mode 0) or the owned grid (grid_mode 1).
dvnr_status mp_decode(dvnr_model m, const float* xyz, int64_t n, int grid_mode, float* out,
                      cudaStream_t s);
// FP16 inference at the samples of rays r0 .. r0+nr-1 of block rb of the
// ray lattice rf, depth-major: out[(k - k0) nr + ray - r0] (nr * rb.nk values).
dvnr_status mp_decode_rays(dvnr_model m, const RayFrame& rf, const RayBlock& rb, int64_t r0, int64_t nr,
                           float* out, cudaStream_t s);
dvnr_status mp_decode_impl(dvnr_model m, const float* xyz, int64_t n, int grid_mode, const RayFrame* rf,
                           const RayBlock* rb, int64_t r0, int64_t nr, float* out, cudaStream_t s,
                           const uint32_t* coords = nullptr);
// Network output y (normalised units, no value range applied) at n given
// fixed-point coordinates (n x 3), FP16 tables and weights.
dvnr_status mp_forward(dvnr_model m, const uint32_t* coords, int64_t n, float* y, cudaStream_t s);
// Backward of the training kernel at n given fixed-point coordinates with the
// upstream gradient dy (n values) instead of a loss, loss scale *scale_dev:
// gradients left (scaled) in m->grad, dL/d(encoding) (unscaled, n x D) in
// dx0 when not null. Synchronises the stream.
dvnr_status mp_backward(dvnr_model m, const uint32_t* coords, const float* dy, int64_t n,
                        const float* scale_dev, float* dx0, cudaStream_t s);

}  // namespace dvnr
