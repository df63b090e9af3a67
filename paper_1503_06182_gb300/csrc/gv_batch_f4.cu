// Batched fill kernels: float, at most 4 axes (4 and 8 events per thread).
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(f4, float, 4)
