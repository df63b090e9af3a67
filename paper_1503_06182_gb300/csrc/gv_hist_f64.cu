// Fill kernels with a histogram of the observable, FP64 form (all integrands).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_HIST_LAUNCHER(double, f64)
