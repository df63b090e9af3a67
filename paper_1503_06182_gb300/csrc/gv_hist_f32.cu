// Fill kernels with a histogram of the observable, FP32 form (all integrands).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_HIST_LAUNCHER(float, f32)
