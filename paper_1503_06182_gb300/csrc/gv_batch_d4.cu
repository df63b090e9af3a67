// Batched fill kernel: double, 4 events per thread.
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(d4, double, 4)
