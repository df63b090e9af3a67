// Batched fill kernels: float, at most 16 axes (4 and 8 events per thread).
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(f16, float, 16)
