// Fill kernels of the LO Drell-Yan integrand, FP32 form.
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_LAUNCHER(launch_fill_dy, GV_DY, float, f32)
