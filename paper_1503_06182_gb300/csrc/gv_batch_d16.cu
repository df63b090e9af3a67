// Batched fill kernels: double, at most 16 axes (4 and 8 events per thread).
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(d16, double, 16)
