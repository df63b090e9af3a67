// Stratified (VEGAS+) fill kernels, FP32 form (all integrands).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_PLUS_LAUNCHER(float, f32)
