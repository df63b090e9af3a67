// Precision dispatch of the fill launchers (the kernels live in
// gv_fill_<integrand>_{f32,f64}.cu).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_DISPATCH(launch_fill_gauss)
GV_DEFINE_FILL_DISPATCH(launch_fill_dy)
GV_DEFINE_FILL_DISPATCH(launch_fill_ee3j)
GV_DEFINE_FILL_DISPATCH(launch_fill_dynlo)
