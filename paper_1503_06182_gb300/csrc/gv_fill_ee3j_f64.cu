// Fill kernels of the e+e- -> q qbar g integrand, FP64 form.
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_LAUNCHER(launch_fill_ee3j, GV_EE3J, double, f64)
