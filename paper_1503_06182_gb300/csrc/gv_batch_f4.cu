// Batched fill kernel: float, 4 events per thread.
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(f4, float, 4)
