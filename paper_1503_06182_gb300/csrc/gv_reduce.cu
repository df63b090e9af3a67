// gv_reduce.cu -- combination of all events of an iteration and the serial
// grid optimisation (Section 2.1: "the grid optimization is not parallelized,
// so that all the results can be combined").
//
// gv_reduce_kernel: each CTA sums the 128-bit tile partials of a contiguous
// range of tiles, aligned to the iteration's scale (max over tiles of E_t,
// an order-free reduction done by the fill kernel), into 192-bit integers and
// adds them to the iteration's accumulators with integer atomics.  Integer
// addition is associative, so the totals do not depend on the number of
// CTAs or their order.  The last CTA to finish (ticket counter, no waiting)
// rounds the totals to FP64, records I_k and sigma_k, updates the stage's
// inverse-variance combination and refines the grid (Lepage's VEGAS, cited
// in Section 2.1): 3-point smoothing, normalisation, compression
// ((1-rho)/(-ln rho))^alpha, redistribution into N equal shares.
#include "gv_integrands.cuh"

struct u192 {
  unsigned long long l0, l1, l2;
};

__device__ __forceinline__ void add192(u192& r, const u192& x) {
  const unsigned long long a0 = r.l0 + x.l0;
  const unsigned long long c0 = a0 < r.l0 ? 1ull : 0ull;
  const unsigned long long t1 = r.l1 + x.l1;
  const unsigned long long c1 = t1 < r.l1 ? 1ull : 0ull;
  const unsigned long long a1 = t1 + c0;
  const unsigned long long c1b = a1 < t1 ? 1ull : 0ull;
  r.l0 = a0;
  r.l1 = a1;
  r.l2 = r.l2 + x.l2 + c1 + c1b;
}

// Arithmetic shift right of a 192-bit two's complement value.
__device__ __forceinline__ u192 sar192(u192 v, int s) {
  const unsigned long long ext = (unsigned long long)((long long)v.l2 >> 63);
  if (s <= 0) return v;
  if (s >= 192) return {ext, ext, ext};
  while (s >= 64) {
    v.l0 = v.l1;
    v.l1 = v.l2;
    v.l2 = ext;
    s -= 64;
  }
  if (s > 0) {
    v.l0 = (v.l0 >> s) | (v.l1 << (64 - s));
    v.l1 = (v.l1 >> s) | (v.l2 << (64 - s));
    v.l2 = (unsigned long long)((long long)v.l2 >> s);
  }
  return v;
}

__device__ __forceinline__ void atomic_add192(unsigned long long* p, const u192& v) {
  const unsigned long long old0 = atomicAdd(p, v.l0);
  const unsigned long long c0 = (old0 + v.l0 < old0) ? 1ull : 0ull;
  const unsigned long long a1 = v.l1 + c0;
  unsigned long long c1 = (a1 < c0) ? 1ull : 0ull;
  if (a1 != 0ull) {
    const unsigned long long old1 = atomicAdd(p + 1, a1);
    c1 += (old1 + a1 < old1) ? 1ull : 0ull;
  }
  const unsigned long long a2 = v.l2 + c1;
  if (a2 != 0ull) atomicAdd(p + 2, a2);
}

// value * 2^q, rounded to nearest (the 192-bit integer is two's complement).
__device__ double u192_to_double(u192 v, int q) {
  const bool neg = (long long)v.l2 < 0;
  if (neg) {
    v.l0 = ~v.l0;
    v.l1 = ~v.l1;
    v.l2 = ~v.l2;
    v.l0 += 1ull;
    const unsigned long long c0 = v.l0 == 0ull ? 1ull : 0ull;
    v.l1 += c0;
    v.l2 += (c0 && v.l1 == 0ull) ? 1ull : 0ull;
  }
  int top;
  if (v.l2)
    top = 191 - __clzll((long long)v.l2);
  else if (v.l1)
    top = 127 - __clzll((long long)v.l1);
  else if (v.l0)
    top = 63 - __clzll((long long)v.l0);
  else
    return 0.0;
  unsigned long long window;
  if (top >= 63) {
    const int sh = top - 63;  // bits below the 64-bit window
    const u192 w = sar192(v, sh);
    window = w.l0;
    bool sticky = false;
    if (sh >= 128) {
      sticky = v.l0 != 0ull || v.l1 != 0ull || (sh > 128 && (v.l2 << (192 - sh)) != 0ull);
    } else if (sh >= 64) {
      sticky = v.l0 != 0ull || (sh > 64 && (v.l1 << (128 - sh)) != 0ull);
    } else if (sh > 0) {
      sticky = (v.l0 << (64 - sh)) != 0ull;
    }
    window |= sticky ? 1ull : 0ull;
  } else {
    window = v.l0 << (63 - top);
  }
  const double m = __ull2double_rn(window);
  const double r = scalbn(m, top - 63 + q);
  return neg ? -r : r;
}

// ---------------------------------------------------------------------------
// Iteration record and stage combination (thread 0 of the last CTA).
// ---------------------------------------------------------------------------
__device__ void mean_sigma(double s1, double s2, long long ncall, double* mean, double* sigma) {
  const double C = (double)ncall;
  const double I = s1 / C;
  const double var = (s2 / C - I * I) / (C - 1.0);
  *mean = I;
  *sigma = var > 0.0 ? sqrt(var) : 0.0;
}

__device__ void combine_stage(const double* per_iter, int stride, int m, GvState* st,
                              bool adjoint) {
  int nzero = 0;
  double zsum = 0.0;
  for (int k = 0; k < m; ++k) {
    const double s = per_iter[k * stride + 1];
    if (!(s > 0.0)) {
      ++nzero;
      zsum += per_iter[k * stride];
    }
  }
  double swt = 0.0, swi = 0.0;
  if (nzero == 0) {
    for (int k = 0; k < m; ++k) {
      const double s = per_iter[k * stride + 1];
      const double wt = 1.0 / (s * s);
      swt += wt;
      swi += wt * per_iter[k * stride];
    }
    const double mean = swi / swt;
    double chi2 = 0.0;
    for (int k = 0; k < m; ++k) {
      const double s = per_iter[k * stride + 1];
      const double dev = per_iter[k * stride] - mean;
      chi2 += dev * dev / (s * s);
    }
    st->integral = mean;
    st->error = 1.0 / sqrt(swt);
    st->chi2 = m > 1 ? chi2 / (m - 1) : 0.0;
  } else {
    st->integral = zsum / nzero;
    st->error = 0.0;
    st->chi2 = 0.0;
  }
  if (adjoint) {
    for (int p = 0; p < GV_NGRAD; ++p) {
      double num = 0.0, den = 0.0, var = 0.0;
      for (int k = 0; k < m; ++k) {
        const double s = per_iter[k * stride + 1];
        const double wt = nzero ? ((s > 0.0) ? 0.0 : 1.0) : 1.0 / (s * s);
        const double G = per_iter[k * stride + 2 + 2 * p];
        const double sG = per_iter[k * stride + 3 + 2 * p];
        num += wt * G;
        den += wt;
        var += wt * wt * sG * sG;
      }
      st->grad[p] = num / den;
      st->grad_err[p] = sqrt(var) / den;
    }
  }
}

// ---------------------------------------------------------------------------
// Grid refinement by the whole CTA.  d: bin sums [ndim][N]; scratch holds
// smoothed/compressed values and cumulative sums.
// ---------------------------------------------------------------------------
__device__ void pack_axis_tables(double* grid, int d, int N, int a_first, int a_last, int tid,
                                 int nthr) {
  const GvGridLayout L{d, N};
  double* e64 = grid + L.off_e64();
  double* wd64 = grid + L.off_wd64();
  double* jac = grid + L.off_jac();
  float* e32 = reinterpret_cast<float*>(grid + L.off_f32_base());
  float* wd32 = e32 + (size_t)d * (N + 1);
  for (int k = tid; k < (a_last - a_first) * (N + 1); k += nthr) {
    const int a = a_first + k / (N + 1), i = k % (N + 1);
    const size_t ie = (size_t)a * (N + 1) + i;
    e32[ie] = (float)e64[ie];
    if (i < N) {
      const double w = e64[ie + 1] - e64[ie];
      wd64[(size_t)a * N + i] = w;
      jac[(size_t)a * N + i] = (double)N * w;
      wd32[(size_t)a * N + i] = (float)w;
    }
  }
}

__device__ void refine_grid(const GvReduceArgs& a, const double* dsum) {
  const int d = a.ndim, N = a.nbins;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nwarps = nthr >> 5;
  double* sm = a.scratch;                        // [d][N]  smoothed, then compressed
  double* cum = a.scratch + (size_t)d * N;       // [d][N+1]
  double* ne = cum + (size_t)d * (N + 1);        // [d][N+1] new edges
  __shared__ double s_total[GV_MAXD];
  double* e64 = a.grid;                          // pack starts with e64
  // 1. smoothing
  for (int k = tid; k < d * N; k += nthr) {
    const int ax = k / N, i = k % N;
    const double* da = dsum + (size_t)ax * N;
    double v;
    if (i == 0)
      v = (da[0] + da[1]) / 2.0;
    else if (i == N - 1)
      v = (da[N - 2] + da[N - 1]) / 2.0;
    else
      v = (da[i - 1] + da[i] + da[i + 1]) / 3.0;
    sm[k] = v;
  }
  __syncthreads();
  // per-axis totals: one warp per axis, fixed lane order, fixed butterfly
  for (int ax = wid; ax < d; ax += nwarps) {
    double t = 0.0;
    for (int i = lane; i < N; i += 32) t += sm[(size_t)ax * N + i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
    if (lane == 0) s_total[ax] = t;
  }
  __syncthreads();
  // 2. normalisation and 3. compression
  for (int k = tid; k < d * N; k += nthr) {
    const int ax = k / N;
    const double total = s_total[ax];
    double r = 0.0;
    if (total > 0.0) {
      const double rho = sm[k] / total;
      if (rho <= 0.0)
        r = 0.0;
      else if (rho >= 1.0)
        r = 1.0;
      else
        r = pow((1.0 - rho) / (-log(rho)), a.alpha);
    }
    sm[k] = r;
  }
  __syncthreads();
  // cumulative sums, one thread per axis, in bin order
  for (int ax = tid; ax < d; ax += nthr) {
    double c = 0.0;
    cum[(size_t)ax * (N + 1)] = 0.0;
    for (int i = 0; i < N; ++i) {
      c += sm[(size_t)ax * N + i];
      cum[(size_t)ax * (N + 1) + i + 1] = c;
    }
  }
  __syncthreads();
  // 4. new edges: edge j sits where the cumulative compressed mass reaches j R/N
  for (int k = tid; k < d * (N + 1); k += nthr) {
    const int ax = k / (N + 1), j = k % (N + 1);
    if (!(s_total[ax] > 0.0)) continue;
    const double* C = cum + (size_t)ax * (N + 1);
    const double* r = sm + (size_t)ax * N;
    const double* e = e64 + (size_t)ax * (N + 1);
    double v;
    if (j == 0) {
      v = 0.0;
    } else if (j == N) {
      v = 1.0;
    } else {
      const double R = C[N];
      const double target = (R / N) * j;
      // first bin i in [0, N-1] with C[i+1] > target (N-1 if none)
      int lo = 0, hi = N - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (C[mid + 1] > target)
          hi = mid;
        else
          lo = mid + 1;
      }
      const int i = lo;
      v = e[i] + (target - C[i]) / r[i] * (e[i + 1] - e[i]);
    }
    ne[k] = v;
  }
  __syncthreads();
  for (int k = tid; k < d * (N + 1); k += nthr) {
    const int ax = k / (N + 1);
    if (s_total[ax] > 0.0) e64[k] = ne[k];
  }
  __syncthreads();
  pack_axis_tables(a.grid, d, N, 0, d, tid, nthr);
}

__device__ void finalize_iteration(const GvReduceArgs& a) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  GvState* st = a.st;
  // totals -> FP64
  for (int k = tid; k < a.nacc; k += nthr) {
    const int ch = k < 2 * a.nch ? (k >> 1) : 0;
    const int pw = k < 2 * a.nch ? ((k & 1) + 1) : 2;
    const int Eg = st->E[ch];
    double v = 0.0;
    if (Eg != GV_EMPTY) {
      u192 t;
      t.l0 = __ldcg(a.acc + 3 * k);
      t.l1 = __ldcg(a.acc + 3 * k + 1);
      t.l2 = __ldcg(a.acc + 3 * k + 2);
      v = u192_to_double(t, pw * Eg - GV_FB);
    }
    a.sums[k] = v;
  }
  __syncthreads();
  if (tid == 0) {
    const int m = st->m;
    const int stride = a.mode ? 2 + 2 * GV_NGRAD : 2;
    double* rec = a.per_iter + (size_t)m * stride;
    mean_sigma(a.sums[0], a.sums[1], a.ncall, &rec[0], &rec[1]);
    if (a.mode) {
      for (int p = 0; p < GV_NGRAD; ++p)
        mean_sigma(a.sums[2 + 2 * p], a.sums[3 + 2 * p], a.ncall, &rec[2 + 2 * p],
                   &rec[3 + 2 * p]);
    }
    st->m = m + 1;
    combine_stage(a.per_iter, stride, m + 1, st, a.mode != 0);
  }
  if (a.adapt && a.has_bins) refine_grid(a, a.sums + 2 * a.nch);
  __syncthreads();
  // reset the accumulators for the next iteration
  for (int k = tid; k < 3 * a.nacc; k += nthr) a.acc[k] = 0ull;
  if (tid == 0) {
    for (int c = 0; c < GV_MAXCH; ++c) st->E[c] = GV_EMPTY;
    st->done = 0;
    st->it = st->it + 1ull;
  }
}

__global__ void __launch_bounds__(256) gv_reduce_kernel(const GvReduceArgs a) {
  const int t0 = blockIdx.x * a.tiles_per_cta;
  const int t1 = min(a.n_tiles, t0 + a.tiles_per_cta);
  for (int k = threadIdx.x; k < a.nacc; k += blockDim.x) {
    const int ch = k < 2 * a.nch ? (k >> 1) : 0;
    const int pw = k < 2 * a.nch ? ((k & 1) + 1) : 2;
    const int Eg = a.st->E[ch];
    if (Eg == GV_EMPTY) continue;
    u192 r = {0ull, 0ull, 0ull};
    for (int t = t0; t < t1; ++t) {
      const int Et = a.tileE[(size_t)t * a.nch + ch];
      if (Et == GV_EMPTY) continue;
      const ulonglong2 v = a.part[(size_t)t * a.nacc + k];
      u192 x = {v.x, v.y, (unsigned long long)((long long)v.y >> 63)};
      x = sar192(x, pw * (Eg - Et));
      add192(r, x);
    }
    if (r.l0 | r.l1 | r.l2) atomic_add192(a.acc + 3 * k, r);
  }
  __threadfence();
  __syncthreads();
  __shared__ int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(&a.st->done, 1) == (int)gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize_iteration(a);
}

// ---------------------------------------------------------------------------
// Setup: derived constants of the integrand and a fresh stage.
// ---------------------------------------------------------------------------
// p[GV_MAXPARAMS - 1] carries the number of user parameters.
__global__ void gv_setup_kernel(int ig, const double* p, double* K, GvState* st, int nacc,
                                unsigned long long* acc) {
  if (threadIdx.x == 0) {
    const int np = (int)p[GV_MAXPARAMS - 1];
    for (int i = 0; i < GV_NCONST; ++i) K[i] = 0.0;
    if (ig == GV_GAUSS) {
      K[GK_INV2S2] = 1.0 / (2.0 * p[0] * p[0]);
    } else if (ig == GV_DY) {
      const double sqrt_s = p[0], MZ = p[1], GZ = p[2], sw2 = p[3], alpha = p[4];
      const double mlo = p[5], mhi = p[6];
      const double s = sqrt_s * sqrt_s;
      const double tau_lo = mlo * mlo / s, tau_hi = mhi * mhi / s;
      const double pi = 3.14159265358979323846;
      K[DK_SQRTS] = sqrt_s;
      K[DK_S] = s;
      K[DK_TAULO] = tau_lo;
      K[DK_L] = log(tau_hi / tau_lo);
      K[DK_MZ2] = MZ * MZ;
      K[DK_GM2] = (GZ * MZ) * (GZ * MZ);
      const double kappa = 1.0 / (4.0 * sw2 * (1.0 - sw2));
      K[DK_KAPPA] = kappa;
      // alpha^2/(4 N_c) * (hbar c)^2 [pb GeV^2] * Jacobians of cos(theta) (2) and phi (2 pi)
      K[DK_PREF] = alpha * alpha / (4.0 * 3.0) * 0.3893794e9 * 2.0 * (2.0 * pi);
      // couplings V = T3 - 2 Q sw2, A = T3; muon Q = -1, T3 = -1/2
      const double Vl = -0.5 + 2.0 * sw2, Al = -0.5, dVl = 2.0;
      double cA0 = 0, cA1 = 0, cA2 = 0, cB1 = 0, cB2 = 0, dA1 = 0, dA2 = 0, dB2 = 0;
      for (int t = 0; t < 2; ++t) {
        const double n = t == 0 ? 2.0 : 3.0;  // u, c  |  d, s, b
        const double Q = t == 0 ? 2.0 / 3.0 : -1.0 / 3.0;
        const double T3 = t == 0 ? 0.5 : -0.5;
        const double Vq = T3 - 2.0 * Q * sw2, Aq = T3, dVq = -2.0 * Q;
        cA0 += n * Q * Q;
        cA1 += n * (-2.0 * Q * Vl * Vq);
        cA2 += n * (Al * Al + Vl * Vl) * (Aq * Aq + Vq * Vq);
        cB1 += n * (-4.0 * Q * Al * Aq);
        cB2 += n * (8.0 * Al * Vl * Aq * Vq);
        dA1 += n * (-2.0 * Q * (dVl * Vq + Vl * dVq));
        dA2 += n * (2.0 * Vl * dVl * (Aq * Aq + Vq * Vq) + (Al * Al + Vl * Vl) * 2.0 * Vq * dVq);
        dB2 += n * (8.0 * Al * Aq * (dVl * Vq + Vl * dVq));
      }
      K[DK_CA0] = cA0;
      K[DK_CA1] = cA1;
      K[DK_CA2] = cA2;
      K[DK_CB1] = cB1;
      K[DK_CB2] = cB2;
      K[DK_A] = p[7];
      K[DK_B] = p[8];
      K[DK_NORM] = 0.2 * p[9] * p[9];
      K[DK_MZ] = MZ;
      K[DK_GZ] = GZ;
      K[DK_DKAPPA] = -kappa * (1.0 - 2.0 * sw2) / (sw2 * (1.0 - sw2));
      K[DK_DCA1] = dA1;
      K[DK_DCA2] = dA2;
      K[DK_DCB2] = dB2;
    } else if (ig == GV_EE3J) {
      const double Q = np > 1 ? p[1] : 91.1876;
      K[EK_YCUT] = p[0];
      K[EK_Q] = Q;
      K[EK_INVQ2] = 1.0 / (Q * Q);
    }
    st->m = 0;
    st->nonfinite = 0ull;
    st->status = 0;
    st->done = 0;
    for (int c = 0; c < GV_MAXCH; ++c) st->E[c] = GV_EMPTY;
    st->integral = st->error = st->chi2 = 0.0;
    for (int q = 0; q < GV_NGRAD; ++q) st->grad[q] = st->grad_err[q] = 0.0;
  }
  for (int k = threadIdx.x; k < 3 * nacc; k += blockDim.x) acc[k] = 0ull;
}

__global__ void gv_grid_pack_kernel(double* grid, int d, int N) {
  pack_axis_tables(grid, d, N, 0, d, threadIdx.x, blockDim.x);
}

__global__ void gv_rng_words_kernel(unsigned long long seed, uint32_t it, uint32_t batch,
                                    unsigned long long ev0, long long n, int d, uint32_t* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t r[GV_MAXD];
  gv_event_words<GV_MAXD>(seed, it, batch, ev0 + (unsigned long long)j, d, r);
  for (int a = 0; a < d; ++a) out[j * d + a] = r[a];
}

namespace gv {
cudaError_t launch_reduce(const GvReduceArgs& a, int ctas, cudaStream_t s) {
  gv_reduce_kernel<<<ctas, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_setup(int integrand, const double* params, double* kconst, GvState* st,
                         int nacc, unsigned long long* acc, cudaStream_t s) {
  gv_setup_kernel<<<1, 256, 0, s>>>(integrand, params, kconst, st, nacc, acc);
  return cudaGetLastError();
}

cudaError_t launch_grid_pack(int d, int N, double* grid, cudaStream_t s) {
  gv_grid_pack_kernel<<<1, 256, 0, s>>>(grid, d, N);
  return cudaGetLastError();
}

cudaError_t launch_rng_words(unsigned long long seed, uint32_t it, uint32_t batch,
                             unsigned long long ev0, long long n, int d, uint32_t* out,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int thr = 256;
  gv_rng_words_kernel<<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(seed, it, batch, ev0, n, d,
                                                                     out);
  return cudaGetLastError();
}
}  // namespace gv
