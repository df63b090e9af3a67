// gv_combine.cuh -- the iteration record and the inverse-variance
// combination of a stage's iterations (Section 2.1: iterations of event sets
// combined into one estimate), shared by the reduce and the VEGAS+ kernels.
#pragma once
#include "gv_common.cuh"

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// ---------------------------------------------------------------------------
// Iteration record and stage combination.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mean_sigma(double s1, double s2, double inv_c, double inv_cm1,
                                           double* mean, double* sigma) {
  const double I = s1 * inv_c;
  const double var = (s2 * inv_c - I * I) * inv_cm1;
  *mean = I;
  *sigma = var > 0.0 ? sqrt(var) : 0.0;
}

// Inverse-variance combination of the iterations 0..m-1 of a stage by one
// warp (lanes stride over the iterations, fixed butterfly sums); if any
// iteration has zero variance, those alone are averaged with error 0.
static __device__ void combine_stage_warp(const double* per_iter, int stride, int m,
                                          double inv_m1, GvState* st, bool adjoint) {
  const int lane = threadIdx.x & 31;
  if (m == 1 && !adjoint) {
    if (lane == 0) {
      st->integral = per_iter[0];
      st->error = per_iter[1];
      st->chi2 = 0.0;
    }
    return;
  }
  double nz = 0.0;
  for (int k = lane; k < m; k += 32) nz += (per_iter[k * stride + 1] > 0.0) ? 0.0 : 1.0;
  nz = warp_sum_f64(nz);
  double swt = 0.0, swi = 0.0;
  for (int k = lane; k < m; k += 32) {
    const double s = per_iter[k * stride + 1];
    const double wt = nz > 0.0 ? (s > 0.0 ? 0.0 : 1.0) : __drcp_rn(s * s);
    swt += wt;
    swi = fma(wt, per_iter[k * stride], swi);
  }
  swt = warp_sum_f64(swt);
  swi = warp_sum_f64(swi);
  const double inv_swt = __drcp_rn(swt);
  const double mean = swi * inv_swt;
  double chi2 = 0.0;
  if (nz == 0.0)
    for (int k = lane; k < m; k += 32) {
      const double s = per_iter[k * stride + 1];
      const double dev = per_iter[k * stride] - mean;
      chi2 = fma(dev * dev, __drcp_rn(s * s), chi2);
    }
  chi2 = warp_sum_f64(chi2);
  if (lane == 0) {
    st->integral = mean;
    st->error = nz > 0.0 ? 0.0 : rsqrt(swt);
    st->chi2 = (nz > 0.0 || m < 2) ? 0.0 : chi2 * inv_m1;
  }
  if (adjoint) {
    for (int p = 0; p < GV_NGRAD; ++p) {
      double num = 0.0, var = 0.0;
      for (int k = lane; k < m; k += 32) {
        const double s = per_iter[k * stride + 1];
        const double wt = nz > 0.0 ? (s > 0.0 ? 0.0 : 1.0) : __drcp_rn(s * s);
        const double sG = per_iter[k * stride + 3 + 2 * p];
        num = fma(wt, per_iter[k * stride + 2 + 2 * p], num);
        var = fma(wt * wt, sG * sG, var);
      }
      num = warp_sum_f64(num);
      var = warp_sum_f64(var);
      if (lane == 0) {
        st->grad[p] = num * inv_swt;
        st->grad_err[p] = sqrt(var) * inv_swt;
      }
    }
  }
}

