// Fill kernels of the Gaussian integrand, FP32 form.
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_LAUNCHER(launch_fill_gauss, GV_GAUSS, float, f32)
