// Batched fill kernel: float, 8 events per thread.
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(f8, float, 8)
