// Adjoint fill kernels (Drell-Yan gradient).
#include "gv_fill_inst.cuh"

template <typename Real, int EPT, int MAXD>
static cudaError_t gv_launch_adj_t(const GvFillArgs& a, int n_tiles, size_t smem, cudaStream_t s,
                                   bool pdl) {
  auto k = gv_fill_adjoint_kernel<Real, EPT, MAXD>;
  cudaError_t e = gv_prepare(k, smem);
  if (e != cudaSuccess) return e;
  return gv_launch(k, dim3(n_tiles), dim3(GV_TILE / EPT), smem, s, pdl, a);
}

template <typename Real, int MAXD>
static cudaError_t gv_launch_adj_ept(int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                     cudaStream_t s, bool pdl) {
  switch (ept) {
    case 1: return gv_launch_adj_t<Real, 1, MAXD>(a, n_tiles, smem, s, pdl);
    case 2: return gv_launch_adj_t<Real, 2, MAXD>(a, n_tiles, smem, s, pdl);
    case 4: return gv_launch_adj_t<Real, 4, MAXD>(a, n_tiles, smem, s, pdl);
  }
  return cudaErrorInvalidValue;
}

namespace gv {
cudaError_t launch_fill_adjoint(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                                cudaStream_t s, bool pdl) {
  if (a.ndim <= 4)
    return fp32 ? gv_launch_adj_ept<float, 4>(ept, a, n_tiles, smem, s, pdl)
                : gv_launch_adj_ept<double, 4>(ept, a, n_tiles, smem, s, pdl);
  if (a.ndim <= 16)
    return fp32 ? gv_launch_adj_ept<float, 16>(ept, a, n_tiles, smem, s, pdl)
                : gv_launch_adj_ept<double, 16>(ept, a, n_tiles, smem, s, pdl);
  return cudaErrorInvalidValue;
}
}  // namespace gv
