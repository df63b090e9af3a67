// Precision dispatch of the fill launchers (the kernels live in
// gv_fill_<integrand>_{f32,f64}.cu, those with a histogram in gv_hist_{f32,f64}.cu, the
// stratified ones in gv_plusfill_{f32,f64}.cu).
#include "gv_fill_inst.cuh"
GV_DEFINE_FILL_DISPATCH(launch_fill_gauss)
GV_DEFINE_FILL_DISPATCH(launch_fill_dy)
GV_DEFINE_FILL_DISPATCH(launch_fill_ee3j)
GV_DEFINE_FILL_DISPATCH(launch_fill_dynlo)

namespace gv {
cudaError_t launch_fill_hist_f32(int ig, const GvFillArgs& a, int n_tiles, size_t smem,
                                 cudaStream_t s, bool pdl);
cudaError_t launch_fill_hist_f64(int ig, const GvFillArgs& a, int n_tiles, size_t smem,
                                 cudaStream_t s, bool pdl);
cudaError_t launch_fill_hist(int ig, int fp32, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl) {
  return fp32 ? launch_fill_hist_f32(ig, a, n_tiles, smem, s, pdl)
              : launch_fill_hist_f64(ig, a, n_tiles, smem, s, pdl);
}
}  // namespace gv

namespace gv {
cudaError_t launch_fill_plus_f32(int ig, const GvFillArgs& a, int n_tiles, size_t smem,
                                 cudaStream_t s, bool pdl);
cudaError_t launch_fill_plus_f64(int ig, const GvFillArgs& a, int n_tiles, size_t smem,
                                 cudaStream_t s, bool pdl);
cudaError_t launch_fill_plus(int ig, int fp32, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl) {
  return fp32 ? launch_fill_plus_f32(ig, a, n_tiles, smem, s, pdl)
              : launch_fill_plus_f64(ig, a, n_tiles, smem, s, pdl);
}
}  // namespace gv
