// gv_integrands.cuh -- device integrands g(x) on the unit cube.
//
// Each event is mapped to phase-space momenta and weighted by |M|^2 times
// parton densities (Section 2.1: "the individual generation of phase space
// points and subsequent matrix element evaluation"; Section 3.2: 3n-4 phase
// space variables plus two parton fractions per event).  The processes are
// synthetic stand-ins for the paper's H+2 jets, chosen so that their integrals
// are known: a Gaussian product, LO pp -> gamma*/Z -> mu+ mu-, and
// e+e- -> q qbar g.  Real = float is the FP32 integrand form (the Jacobian
// product and all sums stay FP64 in the caller); Real = double the plain
// FP64 form.
//
// The library is compiled with -fmad=false: every fused multiply-add is
// written out with Mt::fma, so the rounding of each event's weight is fixed by
// the source and identical in every kernel that evaluates it (any block size,
// events per thread, batched or not).
#pragma once
#include "gv_common.cuh"
#include "gv_math64.cuh"

// Derived constants (filled by the setup kernel from the user parameters).
// Gaussian
#define GK_INV2S2 0
#define GK_SHIFT 1      // constant subtracted from the product (0 by default)
// Drell-Yan
#define DK_SQRTS 0
#define DK_S 1
#define DK_TAULO 2
#define DK_L 3
#define DK_MZ2 4
#define DK_GM2 5
#define DK_KAPPA 6
#define DK_PREF 7
#define DK_CA0 8
#define DK_CA1 9
#define DK_CA2 10
#define DK_CB1 11
#define DK_CB2 12
#define DK_A 13
#define DK_B 14
#define DK_NORM 15
#define DK_MZ 16
#define DK_GZ 17
#define DK_DKAPPA 18
#define DK_DCA1 19
#define DK_DCA2 20
#define DK_DCB2 21
#define DK_LOGTAULO 22  // ln tau_lo
#define DK_NK 23        // Drell-Yan constants
#define NK_BETA 23      // NLO-shaped stand-in: beta
#define NK_INVI0 24     //   1 / I0(beta)
#define NK_NK 25        //   its constants (the Drell-Yan ones first)
// e+e- -> q qbar g
#define EK_YCUT 0
#define EK_Q 1
#define EK_INVQ2 2

template <typename T>
struct GvMath;

// The FP32 form uses the MUFU-based intrinsics (ex2/lg2/rsqrt/rcp/sin/cos
// with a few ulp of error); the FP64 form the table-driven exp and log of
// gv_math64.cuh (within an ulp, fewer FP64 operations than the library's) and
// the library for the rest.
template <>
struct GvMath<float> {
  __device__ static __forceinline__ float exp(float x) { return __expf(x); }
  __device__ static __forceinline__ float log(float x) { return __logf(x); }
  __device__ static __forceinline__ float sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
  __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  __device__ static __forceinline__ void sincospi(float x, float* s, float* c) {
    __sincosf(3.14159265358979f * x, s, c);
  }
  __device__ static __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
};

template <>
struct GvMath<double> {
  __device__ static __forceinline__ double exp(double x) { return gv_exp64(x); }
  __device__ static __forceinline__ double log(double x) {
    return x > 0.0 && x < INFINITY ? gv_log_pos(x) : ::log(x);
  }
  __device__ static __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  __device__ static __forceinline__ double div(double a, double b) { return a / b; }
  __device__ static __forceinline__ void sincospi(double x, double* s, double* c) {
    ::sincospi(x, s, c);
  }
  __device__ static __forceinline__ double fma(double a, double b, double c) {
    return ::fma(a, b, c);
  }
};

// Constants as the integrand's arithmetic type, loaded once per thread.
template <typename Real, int NC>
struct GvConst {
  static_assert(NC <= GV_NCONST_F32, "constants beyond the FP32 copy");
  Real v[NC];
  // FP64 constants from k[0..NC); the FP32 form reads the FP32 copies that
  // the constants kernel stores after them (no conversions per CTA)
  __device__ __forceinline__ void load(const double* k) {
    if constexpr (sizeof(Real) == 4) {
      const float* kf = reinterpret_cast<const float*>(k + GV_NCONST_F32);
#pragma unroll
      for (int i = 0; i < NC; ++i) v[i] = kf[i];
    } else {
#pragma unroll
      for (int i = 0; i < NC; ++i) v[i] = k[i];
    }
  }
  __device__ __forceinline__ Real operator[](int i) const { return v[i]; }
};

// ---------------------------------------------------------------------------
// Gaussian product minus a constant: g = exp(-sum_a (x_a - 1/2)^2 / (2 sigma^2))
// - shift (shift = 0 unless given: negative weights, as NLO subtractions give).
// ---------------------------------------------------------------------------
template <typename Real, int MAXD>
__device__ __forceinline__ Real gv_gauss(const Real (&x)[MAXD], int d, Real inv2s2, Real shift) {
  Real acc = (Real)0;
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    if (a < d) {
      const Real dx = x[a] - (Real)0.5;
      acc = GvMath<Real>::fma(dx, dx, acc);
    }
  }
  return GvMath<Real>::exp(-acc * inv2s2) - shift;
}

// ---------------------------------------------------------------------------
// LO pp -> gamma*/Z -> mu- mu+ (four variables: tau, rapidity, cos theta, phi).
// The partons and leptons are built as light-cone four-vectors
// (p+ = E + pz, p- = E - pz, px, py), so the invariants shat, that, uhat come
// out without the cancellation of E E' - pz pz' at large rapidity.  The
// matrix element is the LO form alpha^2/(4 shat N_c) [(1 + c^2) A + c B]
// summed over u, d, s, c, b with c = (that - uhat)/shat, and the
// antiquark-from-hadron-1 term taking c -> -c.
// With GRAD the reverse sweep also returns dg/d(M_Z, Gamma_Z, sw2, a, b).
// ---------------------------------------------------------------------------
template <typename Real, bool GRAD, int NC>
__device__ __forceinline__ Real gv_drell_yan(const Real* x, const GvConst<Real, NC>& K,
                                             Real* grad) {
  static_assert(NC >= DK_NK, "Drell-Yan constants");
  using Mt = GvMath<Real>;
  const Real one = (Real)1, two = (Real)2;
  // phase space: ln tau linear in x[0]; x1,2 = sqrt(tau) e^(+-y)
  const Real ltau = Mt::fma(x[0], K[DK_L], K[DK_LOGTAULO]);
  const Real tau = Mt::exp(ltau);
  const Real jac_tau = tau * K[DK_L];
  const Real ymax = (Real)(-0.5) * ltau;
  const Real y = Mt::fma(two, x[1], -one) * ymax;
  const Real jac_y = two * ymax;
  const Real opc = two * x[2];          // 1 + cos theta
  const Real omc = two * (one - x[2]);  // 1 - cos theta
  const Real x1 = Mt::exp(y - ymax), x2 = Mt::exp(-y - ymax);
  const Real omx1 = one - x1, omx2 = one - x2;
  if (!(omx1 > (Real)0) || !(omx2 > (Real)0)) {
    // parton densities vanish at x = 1
    if (GRAD) {
#pragma unroll
      for (int p = 0; p < GV_NGRAD; ++p) grad[p] = (Real)0;
    }
    return (Real)0;
  }
  // momenta as light-cone components (p+, p-): partons x1,2 sqrt(s)/2 (1, 0,
  // 0, +-1); the mu- at angle theta in the dilepton frame, boosted by y:
  // p+ = (sqrt(shat)/2)(1 + cos theta) e^y = (sqrt(s)/2) x1 (1 + cos theta),
  // p- = (sqrt(s)/2) x2 (1 - cos theta).  Its transverse momentum enters none
  // of the invariants of the LO matrix element, so phi is a flat direction.
  const Real hs = (Real)0.5 * K[DK_SQRTS];
  const Real p1p = K[DK_SQRTS] * x1;   // parton 1: (p+, 0)
  const Real p2m = K[DK_SQRTS] * x2;   // parton 2: (0, p-)
  const Real p3p = hs * x1 * opc;      // mu-: (p+, p-)
  const Real p3m = hs * x2 * omc;
  const Real shat = p1p * p2m;          // 2 p1.p2
  const Real that = -p1p * p3m;         // -2 p1.p3
  const Real uhat = -p2m * p3p;         // -2 p2.p3
  const Real inv_shat = Mt::div(one, shat);
  const Real c = (that - uhat) * inv_shat;
  const Real opc2 = Mt::fma(c, c, one);
  // parton luminosities f_q(x1) f_qbar(x2) and f_qbar(x1) f_q(x2):
  // ln(x1 x2) = ln tau, ln((1-x1)(1-x2)) in one log
  const Real lx = ltau;
  const Real l1x = Mt::log(omx1 * omx2);
  const Real common = K[DK_NORM] * Mt::exp(Mt::fma(K[DK_A], lx, K[DK_B] * l1x));
  const Real q1 = (omx1 * omx1) * (omx1 * omx1);
  const Real q2 = (omx2 * omx2) * (omx2 * omx2);
  const Real lf = common * q2, lb = common * q1;
  // gamma/Z propagator factors
  const Real D = shat - K[DK_MZ2];
  const Real den = Mt::fma(D, D, K[DK_GM2]);
  const Real inv_den = Mt::div(one, den);
  const Real chi1 = K[DK_KAPPA] * shat * D * inv_den;
  const Real chi2 = K[DK_KAPPA] * K[DK_KAPPA] * shat * shat * inv_den;
  const Real A = Mt::fma(K[DK_CA2], chi2, Mt::fma(K[DK_CA1], chi1, K[DK_CA0]));
  const Real B = Mt::fma(K[DK_CB2], chi2, K[DK_CB1] * chi1);
  const Real S = Mt::fma((lf + lb) * opc2, A, (lf - lb) * c * B);
  const Real P = jac_tau * jac_y * K[DK_PREF] * inv_shat;
  if (GRAD) {
    // reverse sweep from g = P * S
    const Real Sb = P;
    const Real Ab = Sb * (lf + lb) * opc2;
    const Real Bb = Sb * (lf - lb) * c;
    const Real lfb = Sb * Mt::fma(opc2, A, c * B);
    const Real lbb = Sb * Mt::fma(opc2, A, -(c * B));
    const Real commonb = Mt::fma(lfb, q2, lbb * q1);
    const Real gb_a = commonb * common * lx;
    const Real gb_b = commonb * common * l1x;
    const Real chi1b = Mt::fma(Ab, K[DK_CA1], Bb * K[DK_CB1]);
    const Real chi2b = Mt::fma(Ab, K[DK_CA2], Bb * K[DK_CB2]);
    const Real cA1b = Ab * chi1, cA2b = Ab * chi2, cB2b = Bb * chi2;
    const Real kappab = Mt::fma(chi1b * shat, D * inv_den,
                                chi2b * two * K[DK_KAPPA] * shat * shat * inv_den);
    const Real invb = Mt::fma(chi1b * K[DK_KAPPA], shat * D,
                              chi2b * K[DK_KAPPA] * K[DK_KAPPA] * shat * shat);
    const Real denb = -invb * inv_den * inv_den;
    const Real Db = Mt::fma(chi1b * K[DK_KAPPA], shat * inv_den, denb * two * D);
    const Real MZ = K[DK_MZ], GZ = K[DK_GZ];
    // den = D^2 + GZ^2 MZ^2, D = shat - MZ^2
    grad[0] = Mt::fma(denb * two * GZ, GZ * MZ, -(Db * two * MZ));
    grad[1] = denb * two * GZ * MZ * MZ;
    grad[2] = Mt::fma(kappab, K[DK_DKAPPA],
                      Mt::fma(cA1b, K[DK_DCA1], Mt::fma(cA2b, K[DK_DCA2], cB2b * K[DK_DCB2])));
    grad[3] = gb_a;
    grad[4] = gb_b;
  }
  return P * S;
}

// ---------------------------------------------------------------------------
// NLO-shaped stand-in: the Drell-Yan weight of x_0..x_3 times, for every
// further axis, exp(beta cos(2 pi x_k)) / I0(beta) (each factor integrates to
// 1 over [0,1]).  More axes, more work per event, the same integral.
// ---------------------------------------------------------------------------
template <typename Real, int MAXD>
__device__ __forceinline__ Real gv_dy_nlo(const Real (&x)[MAXD], int d,
                                          const GvConst<Real, NK_NK>& K) {
  using Mt = GvMath<Real>;
  Real g = gv_drell_yan<Real, false>(x, K, nullptr);
  Real f = (Real)1;
#pragma unroll
  for (int a = 4; a < MAXD; ++a) {
    if (a < d) {
      Real sn, cs;
      Mt::sincospi((Real)2 * x[a], &sn, &cs);
      f = f * (Mt::exp(K[NK_BETA] * cs) * K[NK_INVI0]);
    }
  }
  return g * f;
}

// ---------------------------------------------------------------------------
// e+e- -> q qbar g, massless: x1 = u0, x2 = u1, x3 = 2 - x1 - x2; cuts
// y_ij > y_cut on the sampled variables; the event plane is rotated by the
// Euler angles (cos theta = 2 u2 - 1, phi = 2 pi u3, psi = 2 pi u4) and
// |M|^2 = (x1^2 + x2^2)/(y23 y13) is evaluated from the momenta.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Real gv_ee3j(const Real* x, const GvConst<Real, 3>& K) {
  using Mt = GvMath<Real>;
  const Real one = (Real)1, two = (Real)2, half = (Real)0.5;
  const Real x1 = x[0], x2 = x[1];
  const Real ycut = K[EK_YCUT];
  if (!((one - x1) > ycut && (one - x2) > ycut && (x1 + x2 - one) > ycut)) return (Real)0;
  const Real x3 = two - x1 - x2;
  const Real Q = K[EK_Q];
  const Real E1 = half * Q * x1, E2 = half * Q * x2, E3 = half * Q * x3;
  const Real c12 = one - Mt::div(two * (one - x3), x1 * x2);
  const Real s12 = Mt::sqrt(fmax(Mt::fma(-c12, c12, one), (Real)0));
  // event plane: p1 along z, p2 in the x-z plane, p3 balances
  const Real p1[3] = {(Real)0, (Real)0, E1};
  const Real p2[3] = {E2 * s12, (Real)0, E2 * c12};
  const Real p3[3] = {-E2 * s12, (Real)0, -E1 - E2 * c12};
  const Real ct = Mt::fma(two, x[2], -one);
  const Real st = Mt::sqrt(fmax(Mt::fma(-ct, ct, one), (Real)0));
  Real sf, cf, sp, cp;
  Mt::sincospi(two * x[3], &sf, &cf);
  Mt::sincospi(two * x[4], &sp, &cp);
  // R = Rz(phi) Ry(theta) Rz(psi)
  const Real R00 = Mt::fma(cf * ct, cp, -(sf * sp)), R01 = Mt::fma(-(cf * ct), sp, -(sf * cp));
  const Real R02 = cf * st;
  const Real R10 = Mt::fma(sf * ct, cp, cf * sp), R11 = Mt::fma(-(sf * ct), sp, cf * cp);
  const Real R12 = sf * st;
  const Real R20 = -st * cp, R21 = st * sp, R22 = ct;
  Real q1[3], q2[3], q3[3];
#define GV_ROT(out, in)                                             \
  out[0] = Mt::fma(R02, in[2], Mt::fma(R01, in[1], R00 * in[0]));   \
  out[1] = Mt::fma(R12, in[2], Mt::fma(R11, in[1], R10 * in[0]));   \
  out[2] = Mt::fma(R22, in[2], Mt::fma(R21, in[1], R20 * in[0]));
  GV_ROT(q1, p1)
  GV_ROT(q2, p2)
  GV_ROT(q3, p3)
#undef GV_ROT
  const Real inv_q2 = K[EK_INVQ2];
  const Real dot13 = Mt::fma(q1[2], q3[2], Mt::fma(q1[1], q3[1], q1[0] * q3[0]));
  const Real dot23 = Mt::fma(q2[2], q3[2], Mt::fma(q2[1], q3[1], q2[0] * q3[0]));
  const Real y13 = two * Mt::fma(E1, E3, -dot13) * inv_q2;
  const Real y23 = two * Mt::fma(E2, E3, -dot23) * inv_q2;
  const Real xm1 = x1, xm2 = x2;  // 2 E_i / Q
  return Mt::div(Mt::fma(xm1, xm1, xm2 * xm2), y23 * y13);
}
