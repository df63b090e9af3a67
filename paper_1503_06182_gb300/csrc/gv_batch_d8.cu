// Batched fill kernel: double, 8 events per thread.
#include "gv_fill_batch.cuh"
GV_DEFINE_FILL_BATCH(d8, double, 8)
