// Fill kernels of the NLO-shaped Drell-Yan stand-in, FP64 form.
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_LAUNCHER(launch_fill_dynlo, GV_DYNLO, double, f64)
