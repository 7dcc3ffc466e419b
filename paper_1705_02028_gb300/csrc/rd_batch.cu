// rd_batch.cu -- batched form (many independent meshes in one graph launch).
#include "rd_internal.h"

extern "C" int rd_batch_create(int32_t, rd_mesh* const*, const double* const*, const rd_params*, rd_batch** out) {
  if (out) *out = nullptr;
  return RD_ENOTSUP;
}
extern "C" int rd_batch_run(rd_batch*, int32_t) { return RD_ENOTSUP; }
extern "C" int rd_batch_get_state(const rd_batch*, int32_t, double*) { return RD_ENOTSUP; }
extern "C" int rd_batch_get_dt(const rd_batch*, double*) { return RD_ENOTSUP; }
extern "C" void rd_batch_destroy(rd_batch*) {}
