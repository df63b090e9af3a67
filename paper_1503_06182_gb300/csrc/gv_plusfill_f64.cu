// Stratified (VEGAS+) fill kernels, FP64 form (all integrands).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_PLUS_LAUNCHER(double, f64)
