// window.cu -- temporal sliding window of trained models (Sec. 4.2: a window
// operator keeps the models of the most recent time steps and drops the
// oldest when full, so that earlier steps stay available for visualisation
// without caching raw grids).
//
// GB300 layout: a step is the set of partition models of one time step, all
// resident in HBM. Only the newest step keeps full trainable models (FP32
// weights, Adam state): the next step's models are warm-started from them
// (Sec. 3.5 weight caching) and trained as one grouped call, after which the
// previous newest step is frozen to its FP16 parameters and value range
// (2 bytes per parameter). A window of N steps therefore holds N - 1 frozen
// steps and one full step, and its device footprint stops growing once it
// is full (the oldest step's models are freed on every further push).
#include <deque>
#include <new>
#include <vector>

#include "dvnr_internal.cuh"

struct dvnr_window_s {
  int device = 0;
  int32_t n_parts = 0;
  int32_t capacity = 0;
  uint64_t seed = 0;
  std::vector<dvnr_box> boxes;
  std::vector<dvnr_enc_cfg> encs;
  dvnr_mlp_cfg mlp{};
  int64_t pushed = 0;  // time steps pushed so far (the next step's index)
  struct Step {
    int64_t t;
    std::vector<dvnr_model> models;
  };
  std::deque<Step> steps;  // oldest .. newest
};

namespace {

void destroy_step(dvnr_window_s::Step& st) {
  for (dvnr_model m : st.models) dvnr_destroy(m);
  st.models.clear();
}

}  // namespace

extern "C" {

dvnr_status dvnr_window_create(const dvnr_box* boxes, int32_t n_parts, const dvnr_enc_cfg* encs,
                               const dvnr_mlp_cfg* mlp, int32_t capacity, uint64_t seed,
                               dvnr_window* out) {
  if (!out) {
    dvnr::set_error("out is NULL");
    return DVNR_E_INVALID;
  }
  *out = nullptr;
  if (!boxes || !encs || !mlp || n_parts < 1 || capacity < 1) {
    dvnr::set_error("need boxes, encodings, an MLP, n_parts >= 1 and capacity >= 1");
    return DVNR_E_INVALID;
  }
  dvnr_window w = new (std::nothrow) dvnr_window_s();
  if (!w) {
    dvnr::set_error("host allocation failed");
    return DVNR_E_OOM;
  }
  cudaGetDevice(&w->device);
  w->n_parts = n_parts;
  w->capacity = capacity;
  w->seed = seed;
  w->boxes.assign(boxes, boxes + n_parts);
  w->encs.assign(encs, encs + n_parts);
  w->mlp = *mlp;
  *out = w;
  return DVNR_OK;
}

void dvnr_window_destroy(dvnr_window w) {
  if (!w) return;
  for (auto& st : w->steps) destroy_step(st);
  delete w;
}

dvnr_status dvnr_window_push(dvnr_window w, const float* const* vol_dev, const dvnr_train_cfg* cfg,
                             void* stream, float* final_loss_host, int64_t* t_out) {
  dvnr::ApiRange nvtx_("dvnr_window_push");
  if (!w || !vol_dev || !cfg) {
    dvnr::set_error("NULL argument");
    return DVNR_E_INVALID;
  }
  cudaSetDevice(w->device);
  // the new step: fresh models, warm-started from the newest step
  dvnr_window_s::Step st;
  st.t = w->pushed;
  dvnr_status rc = DVNR_OK;
  for (int32_t i = 0; i < w->n_parts && rc == DVNR_OK; ++i) {
    dvnr_model m = nullptr;
    rc = dvnr_create(&w->boxes[(size_t)i], &w->encs[(size_t)i], &w->mlp,
                     w->seed + (uint64_t)i, &m);
    if (rc == DVNR_OK) st.models.push_back(m);
  }
  if (rc == DVNR_OK && !w->steps.empty()) {
    const auto& prev = w->steps.back();
    for (int32_t i = 0; i < w->n_parts && rc == DVNR_OK; ++i)
      rc = dvnr_copy_weights(st.models[(size_t)i], prev.models[(size_t)i], stream);
  }
  if (rc == DVNR_OK)
    rc = dvnr_train(st.models.data(), w->n_parts, vol_dev, cfg, stream, final_loss_host);
  if (rc != DVNR_OK) {
    destroy_step(st);
    return rc;
  }
  // the previous newest step becomes storage-only (unless it is about to
  // leave), then the oldest step leaves a full window
  const bool evict = (int32_t)w->steps.size() == w->capacity;
  if (!w->steps.empty() && !(evict && w->steps.size() == 1))
    for (dvnr_model m : w->steps.back().models)
      if ((rc = dvnr_freeze(m, stream)) != DVNR_OK) {  // a model that fails stays as it was
        destroy_step(st);
        return rc;
      }
  if (evict) {
    destroy_step(w->steps.front());
    w->steps.pop_front();
  }
  w->steps.push_back(std::move(st));
  if (t_out) *t_out = w->pushed;
  w->pushed += 1;
  return DVNR_OK;
}

dvnr_status dvnr_window_range(dvnr_window w, int64_t* t_first, int64_t* t_last) {
  if (!w) {
    dvnr::set_error("window is NULL");
    return DVNR_E_INVALID;
  }
  if (t_first) *t_first = w->steps.empty() ? 0 : w->steps.front().t;
  if (t_last) *t_last = w->steps.empty() ? -1 : w->steps.back().t;
  return DVNR_OK;
}

dvnr_status dvnr_window_model(dvnr_window w, int64_t t, int32_t part, dvnr_model* out) {
  if (!w || !out) {
    dvnr::set_error("NULL argument");
    return DVNR_E_INVALID;
  }
  *out = nullptr;
  if (part < 0 || part >= w->n_parts) {
    dvnr::set_error("part %d out of range [0, %d)", part, w->n_parts);
    return DVNR_E_INVALID;
  }
  for (const auto& st : w->steps)
    if (st.t == t) {
      *out = st.models[(size_t)part];
      return DVNR_OK;
    }
  dvnr::set_error("time step %lld is not in the window", (long long)t);
  return DVNR_E_INVALID;
}

dvnr_status dvnr_window_bytes(dvnr_window w, int64_t* model_bytes, int64_t* device_bytes) {
  if (!w) {
    dvnr::set_error("window is NULL");
    return DVNR_E_INVALID;
  }
  int64_t mb = 0, db = 0;
  for (const auto& st : w->steps)
    for (dvnr_model m : st.models) {
      mb += m->n_params * 2;
      db += (int64_t)m->block_bytes;
    }
  if (model_bytes) *model_bytes = mb;
  if (device_bytes) *device_bytes = db;
  return DVNR_OK;
}

}  // extern "C"
