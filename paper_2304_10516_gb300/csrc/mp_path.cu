// mp_path.cu -- placeholder until the tcgen05 kernels land.
#include "mp_path.cuh"

namespace dvnr {
bool mp_supported(const dvnr_model) { return false; }
void mp_release(dvnr_model) {}
dvnr_status mp_train(dvnr_model*, int, const float* const*, const dvnr_train_cfg*, const AdamHyper&,
                     cudaStream_t) {
  set_error("FP16 path not built");
  return DVNR_E_UNSUPPORTED;
}
dvnr_status mp_train_grad(dvnr_model, const float*, const dvnr_train_cfg*, uint32_t, float,
                          const MpStepDebug&, cudaStream_t) {
  set_error("FP16 path not built");
  return DVNR_E_UNSUPPORTED;
}
dvnr_status mp_decode(dvnr_model, const float*, int64_t, int, float*, cudaStream_t) {
  set_error("FP16 path not built");
  return DVNR_E_UNSUPPORTED;
}
}  // namespace dvnr
