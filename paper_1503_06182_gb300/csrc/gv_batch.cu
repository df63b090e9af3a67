// gv_batch.cu -- batched integrations (persistent fill over a work list).
#include "../../include/vegas.h"

extern "C" {
struct vegas_batch {
  int unused;
};
int vegas_batch_create(int, const int*, const int64_t*, const int*, const double*, const int*, int,
                       uint64_t, int, vegas_batch** out) {
  if (out) *out = nullptr;
  return VEGAS_EINVAL;
}
void vegas_batch_free(vegas_batch*) {}
int vegas_batch_set_option(vegas_batch*, int, double) { return VEGAS_EINVAL; }
int vegas_batch_set_stream(vegas_batch*, void*) { return VEGAS_EINVAL; }
int vegas_batch_iterate(vegas_batch*, int, double*, double*, double*, double*) {
  return VEGAS_EINVAL;
}
int vegas_batch_grid_get(const vegas_batch*, int, double*) { return VEGAS_EINVAL; }
}
