// Batched fill kernels: float, at most 8 axes (4 and 8 events per thread).
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(f8, float, 8)
