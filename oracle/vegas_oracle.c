/*
 * vegas_oracle.c -- plain, slow, FP64 CPU VEGAS.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the GPU
 * path.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library; the two are written separately and agree only through the
 * definitions restated below.
 *
 * What it computes (paper: Abstract; Section 2.1; Section 2.2):
 *   - VEGAS [Lepage 1978, cited in Section 2.1] produces successive iterations
 *     of event sets; after each iteration all events are combined and the
 *     adaptive grid is optimised serially (Section 2.1).
 *   - Every event gets its own group of pseudo-random numbers, so the same
 *     events are produced for any number of threads (Section 2.2).  Here the
 *     group is a Philox4x32-10 block (Salmon et al., SC'11) keyed by the seed
 *     and counted by (event, iteration, batch, block).
 *   - Weights are summed with compensated (Kahan/Neumaier) sums (Section 2.2)
 *     in a fixed order: events in index order inside fixed chunks of
 *     ORACLE_CHUNK events, chunk results in chunk order.  The result is
 *     therefore bit-identical for any OpenMP thread count, which is the
 *     paper's validation invariant (Section 2.2) made exact.
 *
 * The VEGAS steps (Lepage 1978; the paper cites the method without restating
 * it) as restated here:
 *   uniform word r (32 bit) -> bin i = floor(r*N / 2^32), in-bin position
 *   f = ((r*N mod 2^32) + 1/2) / 2^32; x = e_i + f*(e_{i+1}-e_i);
 *   Jacobian J = prod_a N*(e_{a,i+1}-e_{a,i});  weight w = J * g(x).
 *   I_k = sum w / C;  var_k = (sum w^2 / C - I_k^2) / (C-1);
 *   d_{a,i} = sum of w^2 over events whose axis-a bin is i.
 *   Combination over the iterations of one call: inverse-variance weights.
 *   Refinement per axis: 3-point smoothing, normalisation, compression
 *   r = ((1-rho)/(-ln rho))^alpha, redistribution of N equal shares of
 *   sum(r) with linear interpolation inside the old bins.
 *
 * Histograms during integration (the paper's differential distributions, the
 * di-jet mass plots of Section 3.2): each event's weight is also summed into
 * the bin of one observable of the event.  Per iteration and bin,
 * H_kb = sum_{e in b} w / C and V_kb = (sum_{e in b} w^2 / C - H_kb^2)/(C-1);
 * a call's iterations are combined with the integral's weights 1/sigma_k^2,
 * so the bins add up to the combined integral.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (oracle/__init__.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_CHUNK 4096
#define ORACLE_MAX_DIM 16
#define ORACLE_NGRAD 5

enum { OR_GAUSS = 0, OR_DY = 1, OR_EE3J = 2, OR_DYNLO = 3 };
enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

static const double OR_PI = 3.14159265358979323846;
static const double GEV2_TO_PB = 0.3893794e9; /* (hbar c)^2 in pb GeV^2 */
static const double N_COLOURS = 3.0;

int oracle_version(void) { return 1; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Ten rounds; in each round the two multipliers
 * act on words 0 and 2, the high halves are xored with words 1/3 and the
 * round key, and the key is bumped by the Weyl constants between rounds.
 * ---------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t prod0 = (uint64_t)mult0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)mult1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* The group of random words of one event: block j of Philox has counter
 * (event low, event high, iteration, batch<<8 | j) and key (seed low, seed
 * high); its word k drives axis 4j+k. */
void oracle_event_words(uint64_t seed, uint32_t iteration, uint32_t batch,
                        uint64_t event, int ndim, uint32_t* words) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; 4 * j < ndim; ++j) {
    uint32_t ctr[4] = {(uint32_t)event, (uint32_t)(event >> 32), iteration,
                       (batch << 8) | (uint32_t)j};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    for (int k = 0; k < 4 && 4 * j + k < ndim; ++k) words[4 * j + k] = out[k];
  }
}

/* Uniform word -> (bin, position inside the bin).  The bin is the integer
 * part of r*N/2^32 (exact on any hardware); the position is the remaining
 * fraction shifted by half a unit so that it is never 0 or 1. */
void oracle_bin_map(uint32_t r, int nbins, int32_t* bin, double* frac) {
  uint64_t v = (uint64_t)r * (uint64_t)(uint32_t)nbins;
  *bin = (int32_t)(v >> 32);
  *frac = ((double)(uint32_t)v + 0.5) * 0x1p-32;
}

/* The adaptive-grid map of one axis: word r -> x = e_i + f (e_{i+1} - e_i)
 * with Jacobian factor N (e_{i+1} - e_i).  Exported for the tests. */
double oracle_grid_map(const double* edges_axis, int nbins, uint32_t r,
                       double* x) {
  int32_t i;
  double f;
  oracle_bin_map(r, nbins, &i, &f);
  double width = edges_axis[i + 1] - edges_axis[i];
  *x = edges_axis[i] + f * width;
  return nbins * width;
}

/* ------------------------------------------------------------------------
 * Integrands g(x) on [0,1]^ndim, each including its own Jacobian to the
 * physical variables and its cuts.
 * ---------------------------------------------------------------------- */

/* Gaussian product: g = prod_a exp(-(x_a - 1/2)^2 / (2 sigma^2)) - shift.
 * The optional constant shift (default 0) makes weights negative where the
 * product is below it, as subtraction terms do at NLO. */
static double gauss_point(int ndim, const double* x, double sigma,
                          double shift) {
  double g = 1.0;
  for (int a = 0; a < ndim; ++a) {
    double dx = x[a] - 0.5;
    g *= exp(-dx * dx / (2.0 * sigma * sigma));
  }
  return g - shift;
}

/* Drell-Yan helpers.  Fermion couplings in the convention V = T3 - 2 Q sw2,
 * A = T3.  Flavours u, d, s, c, b (two up-type, three down-type); muon
 * Q = -1, T3 = -1/2. */
typedef struct {
  double Q, T3;
} fermion_t;

static const fermion_t DY_QUARKS[5] = {
    {2.0 / 3.0, 0.5},   /* u */
    {-1.0 / 3.0, -0.5}, /* d */
    {-1.0 / 3.0, -0.5}, /* s */
    {2.0 / 3.0, 0.5},   /* c */
    {-1.0 / 3.0, -0.5}, /* b */
};
static const fermion_t DY_MUON = {-1.0, -0.5};

/* A light-cone four-vector: p+ = E + pz, p- = E - pz, and the transverse
 * components.  Dot products of massless vectors are formed from these
 * without the cancellation of E*E' - pz*pz' at large rapidity. */
typedef struct {
  double plus, minus, px, py;
} lc4;

static double lc_dot(lc4 p, lc4 q) {
  return 0.5 * (p.plus * q.minus + p.minus * q.plus) - p.px * q.px -
         p.py * q.py;
}

static void lc_to_cartesian(lc4 p, double* out4) {
  out4[0] = 0.5 * (p.plus + p.minus);
  out4[1] = p.px;
  out4[2] = p.py;
  out4[3] = 0.5 * (p.plus - p.minus);
}

/* Vector and axial couplings of a fermion, and dV/dsw2. */
static void dy_couplings(double sw2, fermion_t f, double* V, double* A,
                         double* dV_ds) {
  *V = f.T3 - 2.0 * f.Q * sw2;
  *A = f.T3;
  *dV_ds = -2.0 * f.Q;
}

/* A_q, B_q of the LO form, and their derivatives with respect to
 * (M_Z, Gamma_Z, sw2) when grad != NULL (grad[0..2] for A, grad[3..5] for B). */
static void dy_AB(fermion_t q, double shat, double MZ, double GZ, double sw2,
                  double* Aout, double* Bout, double* grad) {
  double Vq, Aq, dVq, Vl, Al, dVl;
  dy_couplings(sw2, q, &Vq, &Aq, &dVq);
  dy_couplings(sw2, DY_MUON, &Vl, &Al, &dVl);
  double kappa = 1.0 / (4.0 * sw2 * (1.0 - sw2));
  double M2 = MZ * MZ;
  double D = shat - M2;
  double den = D * D + GZ * GZ * M2;
  double chi1 = kappa * shat * D / den;
  double chi2 = kappa * kappa * shat * shat / den;
  double cA1 = -2.0 * q.Q * Vl * Vq;
  double cA2 = (Al * Al + Vl * Vl) * (Aq * Aq + Vq * Vq);
  double cB1 = -4.0 * q.Q * Al * Aq;
  double cB2 = 8.0 * Al * Vl * Aq * Vq;
  *Aout = q.Q * q.Q + cA1 * chi1 + cA2 * chi2;
  *Bout = cB1 * chi1 + cB2 * chi2;
  if (grad) {
    /* M_Z */
    double dden_dM = -4.0 * MZ * D + 2.0 * GZ * GZ * MZ;
    double dchi1_dM = kappa * shat * (-2.0 * MZ * den - D * dden_dM) / (den * den);
    double dchi2_dM = -kappa * kappa * shat * shat * dden_dM / (den * den);
    /* Gamma_Z */
    double dden_dG = 2.0 * GZ * M2;
    double dchi1_dG = -kappa * shat * D * dden_dG / (den * den);
    double dchi2_dG = -kappa * kappa * shat * shat * dden_dG / (den * den);
    /* sw2 through kappa and the vector couplings */
    double dkappa = -kappa * (1.0 - 2.0 * sw2) / (sw2 * (1.0 - sw2));
    double dchi1_ds = chi1 / kappa * dkappa;
    double dchi2_ds = 2.0 * chi2 / kappa * dkappa;
    double dcA1_ds = -2.0 * q.Q * (dVl * Vq + Vl * dVq);
    double dcA2_ds = (2.0 * Vl * dVl) * (Aq * Aq + Vq * Vq) +
                     (Al * Al + Vl * Vl) * (2.0 * Vq * dVq);
    double dcB2_ds = 8.0 * Al * Aq * (dVl * Vq + Vl * dVq);
    grad[0] = cA1 * dchi1_dM + cA2 * dchi2_dM;
    grad[1] = cA1 * dchi1_dG + cA2 * dchi2_dG;
    grad[2] = dcA1_ds * chi1 + cA1 * dchi1_ds + dcA2_ds * chi2 + cA2 * dchi2_ds;
    grad[3] = cB1 * dchi1_dM + cB2 * dchi2_dM;
    grad[4] = cB1 * dchi1_dG + cB2 * dchi2_dG;
    grad[5] = cB1 * dchi1_ds + dcB2_ds * chi2 + cB2 * dchi2_ds;
  }
}

/* Partonic dsigma/dOmega (GeV^-2) for q qbar -> gamma*-or-Z -> mu- mu+ of one
 * flavour type; c = cosine of the angle between the incoming quark and the
 * outgoing mu- in the partonic rest frame.  Standard LO form:
 * alpha^2/(4 shat N_c) [(1+c^2) A + c B].  Exported for the tests. */
double oracle_dy_dsigma_domega(int up_type, double shat, double c,
                               const double* prm) {
  fermion_t q = up_type ? DY_QUARKS[0] : DY_QUARKS[1];
  double A, B;
  dy_AB(q, shat, prm[1], prm[2], prm[3], &A, &B, NULL);
  double alpha = prm[4];
  return alpha * alpha / (4.0 * shat * N_COLOURS) * ((1.0 + c * c) * A + c * B);
}

/* Toy parton densities: f_q = N x^a (1-x)^b, f_qbar = 0.2 N x^a (1-x)^(b+4). */
static double pdf_q(double x, double a, double b, double N) {
  return N * pow(x, a) * pow(1.0 - x, b);
}
static double pdf_qbar(double x, double a, double b, double N) {
  return 0.2 * N * pow(x, a) * pow(1.0 - x, b + 4.0);
}

/* LO pp -> gamma*-or-Z -> mu- mu+ from four unit variables.
 * prm = (sqrt_s, M_Z, Gamma_Z, sw2, alpha, m_lo, m_hi, a, b, N).
 * Variables: tau = tau_lo (tau_hi/tau_lo)^x0, y = (2 x1 - 1)(-ln tau / 2),
 * cos(theta) = 2 x2 - 1, phi = 2 pi x3, with their Jacobians; x1,2 =
 * sqrt(tau) e^(+-y).  The momenta are built, and the matrix element is
 * evaluated from their invariants.  mom (nullable) receives p1, p2 (incoming
 * partons along +z, -z) and p3 (mu-), p4 (mu+) as (E, px, py, pz).
 * grad (nullable) receives dg/d(M_Z, Gamma_Z, sw2, a, b). */
static double dy_point(const double* x, const double* prm, double* mom,
                       double* grad) {
  const double sqrt_s = prm[0], MZ = prm[1], GZ = prm[2], sw2 = prm[3];
  const double alpha = prm[4], mlo = prm[5], mhi = prm[6];
  const double pa = prm[7], pb = prm[8], pN = prm[9];
  const double s = sqrt_s * sqrt_s;
  const double tau_lo = mlo * mlo / s, tau_hi = mhi * mhi / s;
  const double L = log(tau_hi / tau_lo);

  double tau = tau_lo * exp(x[0] * L);
  double jac_tau = tau * L;
  double ymax = -0.5 * log(tau);
  double y = (2.0 * x[1] - 1.0) * ymax;
  double jac_y = 2.0 * ymax;
  double one_plus_c = 2.0 * x[2];
  double one_minus_c = 2.0 * (1.0 - x[2]);
  double jac_c = 2.0;
  double phi = 2.0 * OR_PI * x[3];
  double jac_phi = 2.0 * OR_PI;

  double rt = sqrt(tau);
  double x1 = rt * exp(y), x2 = rt * exp(-y);
  double shat_sampled = tau * s;
  double k = 0.5 * sqrt(shat_sampled);
  double sin_theta = sqrt(one_plus_c * one_minus_c);
  double ey = exp(y), emy = exp(-y);

  lc4 p1 = {sqrt_s * x1, 0.0, 0.0, 0.0};
  lc4 p2 = {0.0, sqrt_s * x2, 0.0, 0.0};
  lc4 p3 = {k * one_plus_c * ey, k * one_minus_c * emy,
            k * sin_theta * cos(phi), k * sin_theta * sin(phi)};
  lc4 p4 = {k * one_minus_c * ey, k * one_plus_c * emy, -p3.px, -p3.py};
  if (mom) {
    lc_to_cartesian(p1, mom + 0);
    lc_to_cartesian(p2, mom + 4);
    lc_to_cartesian(p3, mom + 8);
    lc_to_cartesian(p4, mom + 12);
  }

  double shat = 2.0 * lc_dot(p1, p2);
  double that = -2.0 * lc_dot(p1, p3);
  double uhat = -2.0 * lc_dot(p2, p3);
  double cstar = (that - uhat) / shat;

  double fq1 = pdf_q(x1, pa, pb, pN), fqb1 = pdf_qbar(x1, pa, pb, pN);
  double fq2 = pdf_q(x2, pa, pb, pN), fqb2 = pdf_qbar(x2, pa, pb, pN);
  double lumi_fwd = fq1 * fqb2; /* quark from hadron 1 */
  double lumi_bwd = fqb1 * fq2; /* antiquark from hadron 1: angle is pi-theta */

  double pref = alpha * alpha / (4.0 * shat * N_COLOURS);
  double sum = 0.0, dsum[3] = {0.0, 0.0, 0.0};
  for (int f = 0; f < 5; ++f) {
    double A, B, dAB[6];
    dy_AB(DY_QUARKS[f], shat, MZ, GZ, sw2, &A, &B, grad ? dAB : NULL);
    double term_fwd = (1.0 + cstar * cstar) * A + cstar * B;
    double term_bwd = (1.0 + cstar * cstar) * A - cstar * B;
    sum += lumi_fwd * term_fwd + lumi_bwd * term_bwd;
    if (grad) {
      for (int p = 0; p < 3; ++p) {
        double dA = dAB[p], dB = dAB[3 + p];
        dsum[p] += lumi_fwd * ((1.0 + cstar * cstar) * dA + cstar * dB) +
                   lumi_bwd * ((1.0 + cstar * cstar) * dA - cstar * dB);
      }
    }
  }
  double jac = jac_tau * jac_y * jac_c * jac_phi;
  double g = jac * pref * sum * GEV2_TO_PB;
  if (grad) {
    grad[0] = jac * pref * dsum[0] * GEV2_TO_PB;
    grad[1] = jac * pref * dsum[1] * GEV2_TO_PB;
    grad[2] = jac * pref * dsum[2] * GEV2_TO_PB;
    /* Every parton-density product carries x1^a x2^a and (1-x1)^b (1-x2)^b. */
    grad[3] = (log(x1) + log(x2)) * g;
    grad[4] = (log(1.0 - x1) + log(1.0 - x2)) * g;
  }
  return g;
}

/* e+e- -> q qbar g, massless: x1 = u0, x2 = u1, x3 = 2 - x1 - x2; cuts
 * y_ij > y_cut on the sampled variables; the event is oriented by the Euler
 * angles cos(theta) = 2 u2 - 1, phi = 2 pi u3, psi = 2 pi u4 (unit volume).
 * |M|^2 = (x1^2 + x2^2) / ((1 - x1)(1 - x2)), evaluated from the momenta as
 * x_i = 2 E_i / Q, 1 - x1 = y23, 1 - x2 = y13, y_ij = 2 p_i.p_j / Q^2.
 * prm = (y_cut [, sqrt_s]).  mom (nullable): p1, p2, p3 as (E, px, py, pz). */
static double ee3j_point(const double* x, const double* prm, int nparams,
                         double* mom) {
  const double ycut = prm[0];
  const double Q = nparams > 1 ? prm[1] : 91.1876;
  double x1 = x[0], x2 = x[1], x3 = 2.0 - x1 - x2;
  if (mom) memset(mom, 0, 12 * sizeof(double));
  if (!((1.0 - x1) > ycut && (1.0 - x2) > ycut && (x1 + x2 - 1.0) > ycut))
    return 0.0;
  double E1 = 0.5 * Q * x1, E2 = 0.5 * Q * x2, E3 = 0.5 * Q * x3;
  double c12 = 1.0 - 2.0 * (1.0 - x3) / (x1 * x2);
  double s12 = sqrt(fmax(0.0, 1.0 - c12 * c12));
  /* event plane: p1 along z, p2 in the x-z plane, p3 balances */
  double p[3][4] = {{E1, 0.0, 0.0, E1},
                    {E2, E2 * s12, 0.0, E2 * c12},
                    {E3, -E2 * s12, 0.0, -E1 - E2 * c12}};
  double ct = 2.0 * x[2] - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double phi = 2.0 * OR_PI * x[3], psi = 2.0 * OR_PI * x[4];
  double cf = cos(phi), sf = sin(phi), cp = cos(psi), sp = sin(psi);
  /* R = Rz(phi) Ry(theta) Rz(psi) */
  double R[3][3] = {
      {cf * ct * cp - sf * sp, -cf * ct * sp - sf * cp, cf * st},
      {sf * ct * cp + cf * sp, -sf * ct * sp + cf * cp, sf * st},
      {-st * cp, st * sp, ct}};
  double q[3][4];
  for (int i = 0; i < 3; ++i) {
    q[i][0] = p[i][0];
    for (int r = 0; r < 3; ++r)
      q[i][1 + r] = R[r][0] * p[i][1] + R[r][1] * p[i][2] + R[r][2] * p[i][3];
  }
  if (mom)
    for (int i = 0; i < 3; ++i)
      for (int m = 0; m < 4; ++m) mom[4 * i + m] = q[i][m];
  double Q2 = Q * Q;
#define DOT4(a, b) (a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3])
  double y13 = 2.0 * DOT4(q[0], q[2]) / Q2;
  double y23 = 2.0 * DOT4(q[1], q[2]) / Q2;
#undef DOT4
  double xm1 = 2.0 * q[0][0] / Q, xm2 = 2.0 * q[1][0] / Q;
  return (xm1 * xm1 + xm2 * xm2) / (y23 * y13);
}

/* NLO-shaped stand-in for the paper's 13-dimensional NLO integral (Section
 * 3.2): the LO Drell-Yan weight of the first four variables times, for every
 * further axis k, the factor h(x_k) = exp(beta cos(2 pi x_k)) / I0(beta).
 * Each factor integrates to 1 over [0,1] (I0, the modified Bessel function of
 * order 0, is the integral of exp(beta cos(2 pi u)) by definition), so the
 * integral is the Drell-Yan cross section for any ndim and beta; the extra
 * axes only add work per event.  Parameters: the ten Drell-Yan ones, beta. */
static double bessel_i0(double b) {
  /* I0(b) = sum_k ((b/2)^k / k!)^2 */
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= (0.25 * b * b) / ((double)k * (double)k);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return sum;
}

static double dynlo_point(int ndim, const double* x, const double* prm, double* mom) {
  double g = dy_point(x, prm, mom, NULL);
  const double beta = prm[10];
  const double i0 = bessel_i0(beta);
  for (int k = 4; k < ndim; ++k) g *= exp(beta * cos(2.0 * OR_PI * x[k])) / i0;
  return g;
}

static int check_integrand(int id, int ndim, int nparams) {
  switch (id) {
    case OR_GAUSS:
      return (ndim >= 1 && (nparams == 1 || nparams == 2)) ? OR_OK : OR_EINVAL;
    case OR_DY: return (ndim >= 4 && nparams == 10) ? OR_OK : OR_EINVAL;
    case OR_EE3J:
      return (ndim >= 5 && (nparams == 1 || nparams == 2)) ? OR_OK : OR_EINVAL;
    case OR_DYNLO: return (ndim >= 4 && nparams == 11) ? OR_OK : OR_EINVAL;
    default: return OR_EINVAL;
  }
}

static double integrand_point(int id, int ndim, const double* x,
                              const double* prm, int nparams, double* mom,
                              double* grad) {
  switch (id) {
    case OR_GAUSS: return gauss_point(ndim, x, prm[0], nparams > 1 ? prm[1] : 0.0);
    case OR_DY: return dy_point(x, prm, mom, grad);
    case OR_EE3J: return ee3j_point(x, prm, nparams, mom);
    case OR_DYNLO: return dynlo_point(ndim, x, prm, mom);
  }
  return 0.0;
}

/* The histogram observable of an event at x (Section 3.2's differential
 * distributions):
 *   Gauss: x_0;
 *   Drell-Yan (LO and the NLO-shaped stand-in): the dilepton invariant mass
 *     m_ll in GeV; at LO the pair carries the whole partonic energy, so
 *     m_ll^2 = shat = tau s with tau as in dy_point;
 *   e+e- -> q qbar g: the thrust, which for three massless partons is the
 *     largest energy fraction max(x1, x2, x3) with x3 = 2 - x1 - x2. */
static double observable(int id, const double* x, const double* prm) {
  switch (id) {
    case OR_GAUSS: return x[0];
    case OR_DY:
    case OR_DYNLO: {
      const double sqrt_s = prm[0], mlo = prm[5], mhi = prm[6];
      const double s = sqrt_s * sqrt_s;
      const double tau_lo = mlo * mlo / s, tau_hi = mhi * mhi / s;
      const double tau = tau_lo * exp(x[0] * log(tau_hi / tau_lo));
      return sqrt(tau * s);
    }
    case OR_EE3J: {
      const double x1 = x[0], x2 = x[1], x3 = 2.0 - x1 - x2;
      double t = x1 > x2 ? x1 : x2;
      return t > x3 ? t : x3;
    }
  }
  return 0.0;
}

int oracle_observable(int id, int ndim, const double* x, const double* prm,
                      int nparams, double* obs) {
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  *obs = observable(id, x, prm);
  return OR_OK;
}

/* Bin of an observable value among nh equal bins over [lo, hi), with
 * underflow 0 and overflow nh + 1 (a value that is not a number counts as
 * underflow); invw = nh / (hi - lo).  The position is (v - lo) * invw in
 * FP64, truncated. */
static int hist_bin(double v, double lo, double invw, int nh) {
  if (!(v >= lo)) return 0;
  double t = (v - lo) * invw;
  if (!(t < (double)nh)) return nh + 1;
  return 1 + (int)t;
}

int oracle_hist_bin(double v, int nh, double lo, double hi) {
  return hist_bin(v, lo, (double)nh / (hi - lo), nh);
}

/* g at a point of the unit cube (exported for the tests). */
int oracle_integrand(int id, int ndim, const double* x, const double* prm,
                     int nparams, double* g, double* mom, double* grad) {
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  if (grad && id != OR_DY) return OR_EINVAL;
  *g = integrand_point(id, ndim, x, prm, nparams, mom, grad);
  return OR_OK;
}

/* One event: words -> bins -> x and J -> w = J g.  Exported for the tests,
 * which also compare single GPU events against it. */
static double event_weight(int id, int ndim, int nbins, const double* edges,
                           const double* prm, int nparams, uint64_t seed,
                           uint32_t it, uint32_t batch, uint64_t ev,
                           int32_t* bins, double* xout, double* grad) {
  uint32_t words[ORACLE_MAX_DIM];
  double x[ORACLE_MAX_DIM];
  oracle_event_words(seed, it, batch, ev, ndim, words);
  double J = 1.0;
  for (int a = 0; a < ndim; ++a) {
    int32_t i;
    double f;
    oracle_bin_map(words[a], nbins, &i, &f);
    const double* e = edges + (size_t)a * (nbins + 1);
    double width = e[i + 1] - e[i];
    x[a] = e[i] + f * width;
    J *= nbins * width;
    if (bins) bins[a] = i;
  }
  if (xout) memcpy(xout, x, ndim * sizeof(double));
  double g = integrand_point(id, ndim, x, prm, nparams, NULL, grad);
  if (grad)
    for (int p = 0; p < ORACLE_NGRAD; ++p) grad[p] *= J;
  return J * g;
}

int oracle_event(int id, int ndim, int nbins, const double* edges,
                 const double* prm, int nparams, uint64_t seed, uint32_t it,
                 uint32_t batch, uint64_t ev, double* w, int32_t* bins,
                 double* x) {
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  if (ndim > ORACLE_MAX_DIM || nbins < 2) return OR_EINVAL;
  *w = event_weight(id, ndim, nbins, edges, prm, nparams, seed, it, batch, ev,
                    bins, x, NULL);
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * Compensated summation (Neumaier's variant of Kahan's; Section 2.2).
 * ---------------------------------------------------------------------- */
typedef struct {
  double s, c;
} csum_t;

static void csum_add(csum_t* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

static double csum_value(const csum_t* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------
 * Combination of the iterations of one call, and grid refinement.
 * ---------------------------------------------------------------------- */

/* Inverse-variance combination.  If any iteration has zero variance, the
 * zero-variance iterations alone are averaged and the error is 0. */
void oracle_combine(int m, const double* Ik, const double* sk, double* integral,
                    double* error, double* chi2dof) {
  int nzero = 0;
  double zsum = 0.0;
  for (int k = 0; k < m; ++k)
    if (!(sk[k] > 0.0)) {
      ++nzero;
      zsum += Ik[k];
    }
  if (nzero > 0) {
    *integral = zsum / nzero;
    *error = 0.0;
    *chi2dof = 0.0;
    return;
  }
  double swt = 0.0, swi = 0.0;
  for (int k = 0; k < m; ++k) {
    double wt = 1.0 / (sk[k] * sk[k]);
    swt += wt;
    swi += wt * Ik[k];
  }
  double mean = swi / swt;
  double chi2 = 0.0;
  for (int k = 0; k < m; ++k) {
    double dev = Ik[k] - mean;
    chi2 += dev * dev / (sk[k] * sk[k]);
  }
  *integral = mean;
  *error = 1.0 / sqrt(swt);
  *chi2dof = m > 1 ? chi2 / (m - 1) : 0.0;
}

/* Grid refinement from the per-bin sums d (ndim x nbins, row = axis).
 * Axes whose sums are all zero are left unchanged. */
int oracle_refine(int ndim, int nbins, double alpha, const double* d,
                  double* edges) {
  if (ndim < 1 || nbins < 2) return OR_EINVAL;
  const int N = nbins;
  double* sm = (double*)malloc(sizeof(double) * N);
  double* r = (double*)malloc(sizeof(double) * N);
  double* ne = (double*)malloc(sizeof(double) * (N + 1));
  if (!sm || !r || !ne) {
    free(sm);
    free(r);
    free(ne);
    return OR_ENOMEM;
  }
  for (int a = 0; a < ndim; ++a) {
    const double* da = d + (size_t)a * N;
    double* e = edges + (size_t)a * (N + 1);
    /* 1. smoothing with the neighbouring bins */
    sm[0] = (da[0] + da[1]) / 2.0;
    for (int i = 1; i < N - 1; ++i) sm[i] = (da[i - 1] + da[i] + da[i + 1]) / 3.0;
    sm[N - 1] = (da[N - 2] + da[N - 1]) / 2.0;
    double total = 0.0;
    for (int i = 0; i < N; ++i) total += sm[i];
    if (!(total > 0.0)) continue;
    /* 2. normalisation and 3. compression */
    double R = 0.0;
    for (int i = 0; i < N; ++i) {
      double rho = sm[i] / total;
      if (rho <= 0.0)
        r[i] = 0.0;
      else if (rho >= 1.0)
        r[i] = 1.0;
      else
        r[i] = pow((1.0 - rho) / (-log(rho)), alpha);
      R += r[i];
    }
    /* 4. N equal shares of R, each old bin holding r_i spread uniformly */
    double share = R / N;
    ne[0] = 0.0;
    ne[N] = 1.0;
    int i = 0;
    double cum = 0.0; /* sum of r over the old bins before bin i */
    for (int j = 1; j < N; ++j) {
      double target = share * j;
      while (i < N - 1 && cum + r[i] <= target) {
        cum += r[i];
        ++i;
      }
      ne[j] = e[i] + (target - cum) / r[i] * (e[i + 1] - e[i]);
    }
    memcpy(e, ne, sizeof(double) * (N + 1));
  }
  free(sm);
  free(r);
  free(ne);
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * One VEGAS iteration: all events, combined in a fixed order.
 * channels: 1 (w) for the forward pass, 1 + ORACLE_NGRAD for the adjoint.
 * sums (out): per channel (sum v, sum v^2), then ndim*nbins bin sums of w^2
 * when want_bins.
 * ---------------------------------------------------------------------- */
static int iteration_sums(int id, int ndim, int nbins, const double* edges,
                          const double* prm, int nparams, uint64_t seed,
                          uint32_t it, uint32_t batch, int64_t ncall,
                          int nch, int want_bins, int nh, double h_lo,
                          double h_invw, double* sums, int64_t* nonfinite) {
  const int nbin_acc = want_bins ? ndim * nbins : 0;
  const int hb = nh > 0 ? nh + 2 : 0; /* histogram bins incl. under/overflow */
  const int h0 = 2 * nch + nbin_acc;  /* sum w of bin b at h0 + b, sum w^2 at h0 + hb + b */
  const int nacc = h0 + 2 * hb;
  const int64_t nchunks = (ncall + ORACLE_CHUNK - 1) / ORACLE_CHUNK;
  csum_t* total = (csum_t*)calloc((size_t)nacc, sizeof(csum_t));
  if (!total) return OR_ENOMEM;
  int64_t bad_total = 0;
  int fail = 0;
#pragma omp parallel
  {
    csum_t* part = (csum_t*)malloc(sizeof(csum_t) * (size_t)nacc);
    if (!part) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for ordered schedule(static, 1)
    for (int64_t ch = 0; ch < nchunks; ++ch) {
      int64_t bad = 0;
      if (part) {
        memset(part, 0, sizeof(csum_t) * (size_t)nacc);
        int64_t e0 = ch * ORACLE_CHUNK;
        int64_t e1 = e0 + ORACLE_CHUNK < ncall ? e0 + ORACLE_CHUNK : ncall;
        for (int64_t ev = e0; ev < e1; ++ev) {
          int32_t bins[ORACLE_MAX_DIM];
          double grad[ORACLE_NGRAD];
          double v[1 + ORACLE_NGRAD];
          double x[ORACLE_MAX_DIM];
          v[0] = event_weight(id, ndim, nbins, edges, prm, nparams, seed, it,
                              batch, (uint64_t)ev, bins, x,
                              nch > 1 ? grad : NULL);
          for (int c = 1; c < nch; ++c) v[c] = grad[c - 1];
          int finite = 1;
          for (int c = 0; c < nch; ++c) finite &= isfinite(v[c]) ? 1 : 0;
          if (!finite) {
            ++bad;
            continue; /* a non-finite event contributes nothing */
          }
          for (int c = 0; c < nch; ++c) {
            csum_add(&part[2 * c], v[c]);
            csum_add(&part[2 * c + 1], v[c] * v[c]);
          }
          if (want_bins) {
            double w2 = v[0] * v[0];
            for (int a = 0; a < ndim; ++a)
              csum_add(&part[2 * nch + a * nbins + bins[a]], w2);
          }
          if (hb) {
            int b = hist_bin(observable(id, x, prm), h_lo, h_invw, nh);
            csum_add(&part[h0 + b], v[0]);
            csum_add(&part[h0 + hb + b], v[0] * v[0]);
          }
        }
      }
#pragma omp ordered
      {
        if (part)
          for (int k = 0; k < nacc; ++k) csum_add(&total[k], csum_value(&part[k]));
        bad_total += bad;
      }
    }
    free(part);
  }
  if (fail) {
    free(total);
    return OR_ENOMEM;
  }
  for (int k = 0; k < nacc; ++k) sums[k] = csum_value(&total[k]);
  if (nonfinite) *nonfinite = bad_total;
  free(total);
  return OR_OK;
}

static void mean_sigma(double s1, double s2, int64_t ncall, double* mean,
                       double* sigma) {
  double C = (double)ncall;
  double I = s1 / C;
  double var = (s2 / C - I * I) / (C - 1.0);
  *mean = I;
  *sigma = var > 0.0 ? sqrt(var) : 0.0;
}

/* Combination of the histograms of the m iterations of one call, bin by bin,
 * with the weights of the integral (oracle_combine): 1/sigma_k^2, so that
 * the bins of the combined histogram add up to the combined integral; if any
 * sigma_k is 0, the zero-variance iterations alone, with equal weights.
 * H, V: m x hb (row = iteration) bin estimates and their variances;
 * value, error: hb each.
 *   value_b = sum_k u_k H_kb / sum_k u_k,
 *   error_b = sqrt(sum_k u_k^2 V_kb) / sum_k u_k. */
void oracle_hist_combine(int m, int hb, const double* sk, const double* H,
                         const double* V, double* value, double* error) {
  int nzero = 0;
  for (int k = 0; k < m; ++k)
    if (!(sk[k] > 0.0)) ++nzero;
  double W = 0.0;
  for (int k = 0; k < m; ++k) {
    if (nzero > 0)
      W += sk[k] > 0.0 ? 0.0 : 1.0;
    else
      W += 1.0 / (sk[k] * sk[k]);
  }
  for (int b = 0; b < hb; ++b) {
    double sv = 0.0, se = 0.0;
    for (int k = 0; k < m; ++k) {
      double u;
      if (nzero > 0)
        u = sk[k] > 0.0 ? 0.0 : 1.0;
      else
        u = 1.0 / (sk[k] * sk[k]);
      sv += u * H[(size_t)k * hb + b];
      se += u * u * V[(size_t)k * hb + b];
    }
    value[b] = sv / W;
    error[b] = sqrt(se) / W;
  }
}

/* itmx iterations of one call ("stage").  *iteration is the global
 * iteration counter (the Philox counter word), advanced by itmx.  edges
 * (ndim x (nbins+1)) is refined after every iteration when adapt != 0.
 * per_iter (nullable): itmx x (I_k, sigma_k).  last_sums (nullable): the sums
 * of the last iteration, (sum w, sum w^2, d[ndim*nbins]).
 * Histogram (nh > 0 bins over [lo, hi), plus underflow and overflow, so
 * hb = nh + 2 entries): hist_value, hist_error (hb each, nullable) the
 * combined histogram; hist_last (nullable, 2 hb) the last iteration's
 * sum w then sum w^2 per bin.
 * Returns the number of non-finite events seen through *nonfinite. */
int oracle_iterate_hist(int ndim, int nbins, uint64_t seed, uint32_t batch,
                        uint64_t* iteration, int64_t ncall, int itmx, int id,
                        const double* prm, int nparams, double alpha, int adapt,
                        double* edges, int nh, double lo, double hi,
                        double* integral, double* error, double* chi2dof,
                        double* per_iter, double* last_sums, double* hist_value,
                        double* hist_error, double* hist_last,
                        int64_t* nonfinite) {
  if (ndim < 1 || ndim > ORACLE_MAX_DIM || nbins < 2 || ncall < 2 || itmx < 1)
    return OR_EINVAL;
  if (nh < 0 || (nh > 0 && !(hi > lo))) return OR_EINVAL;
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  const int hb = nh > 0 ? nh + 2 : 0;
  const int nd = 2 + ndim * nbins;
  const int nacc = nd + 2 * hb;
  const double invw = nh > 0 ? (double)nh / (hi - lo) : 0.0;
  const double C = (double)ncall;
  double* sums = (double*)malloc(sizeof(double) * nacc);
  double* Ik = (double*)malloc(sizeof(double) * itmx);
  double* sk = (double*)malloc(sizeof(double) * itmx);
  double* H = (double*)malloc(sizeof(double) * ((size_t)itmx * hb + 1));
  double* V = (double*)malloc(sizeof(double) * ((size_t)itmx * hb + 1));
  if (!sums || !Ik || !sk || !H || !V) {
    free(sums);
    free(Ik);
    free(sk);
    free(H);
    free(V);
    return OR_ENOMEM;
  }
  int64_t bad_all = 0;
  for (int k = 0; k < itmx; ++k) {
    uint32_t it = (uint32_t)(*iteration);
    int64_t bad = 0;
    st = iteration_sums(id, ndim, nbins, edges, prm, nparams, seed, it, batch,
                        ncall, 1, 1, nh, lo, invw, sums, &bad);
    if (st) break;
    bad_all += bad;
    *iteration += 1;
    mean_sigma(sums[0], sums[1], ncall, &Ik[k], &sk[k]);
    if (per_iter) {
      per_iter[2 * k] = Ik[k];
      per_iter[2 * k + 1] = sk[k];
    }
    for (int b = 0; b < hb; ++b) {
      /* the bin's share of the iteration estimate and its variance */
      double h = sums[nd + b] / C;
      double v = (sums[nd + hb + b] / C - h * h) / (C - 1.0);
      H[(size_t)k * hb + b] = h;
      V[(size_t)k * hb + b] = v > 0.0 ? v : 0.0;
    }
    if (k == itmx - 1) {
      if (last_sums) memcpy(last_sums, sums, sizeof(double) * nd);
      if (hist_last && hb) memcpy(hist_last, sums + nd, sizeof(double) * 2 * hb);
    }
    if (adapt) oracle_refine(ndim, nbins, alpha, sums + 2, edges);
  }
  if (!st) {
    oracle_combine(itmx, Ik, sk, integral, error, chi2dof);
    if (hb && hist_value && hist_error)
      oracle_hist_combine(itmx, hb, sk, H, V, hist_value, hist_error);
  }
  if (nonfinite) *nonfinite = bad_all;
  free(sums);
  free(Ik);
  free(sk);
  free(H);
  free(V);
  return st;
}

int oracle_iterate(int ndim, int nbins, uint64_t seed, uint32_t batch,
                   uint64_t* iteration, int64_t ncall, int itmx, int id,
                   const double* prm, int nparams, double alpha, int adapt,
                   double* edges, double* integral, double* error,
                   double* chi2dof, double* per_iter, double* last_sums,
                   int64_t* nonfinite) {
  return oracle_iterate_hist(ndim, nbins, seed, batch, iteration, ncall, itmx,
                             id, prm, nparams, alpha, adapt, edges, 0, 0.0, 0.0,
                             integral, error, chi2dof, per_iter, last_sums, NULL,
                             NULL, NULL, nonfinite);
}

/* Gradient of the Drell-Yan cross section with respect to
 * (M_Z, Gamma_Z, sw2, a, b) on a frozen grid: itmx iterations on the same
 * event streams as a forward call with the same iteration counter.  Per
 * iteration G_kp = mean of dw/dtheta_p; the iterations are combined with
 * the weights 1/sigma_k^2 of the forward estimate (their own dependence on
 * theta is not differentiated).
 * per_iter (nullable): itmx x (I_k, sigma_k); per_iter_grad (nullable):
 * itmx x ORACLE_NGRAD x (G_kp, sigma_Gkp). */
int oracle_adjoint(int ndim, int nbins, uint64_t seed, uint32_t batch,
                   uint64_t* iteration, int64_t ncall, int itmx, int id,
                   const double* prm, int nparams, const double* edges,
                   double* grad, double* grad_err, double* integral,
                   double* error, double* per_iter, double* per_iter_grad) {
  if (id != OR_DY) return OR_EINVAL;
  if (ndim < 4 || ndim > ORACLE_MAX_DIM || nbins < 2 || ncall < 2 || itmx < 1)
    return OR_EINVAL;
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  const int nch = 1 + ORACLE_NGRAD;
  double sums[2 * (1 + ORACLE_NGRAD)];
  double* Ik = (double*)malloc(sizeof(double) * itmx);
  double* sk = (double*)malloc(sizeof(double) * itmx);
  double* Gk = (double*)malloc(sizeof(double) * itmx * ORACLE_NGRAD);
  double* sGk = (double*)malloc(sizeof(double) * itmx * ORACLE_NGRAD);
  if (!Ik || !sk || !Gk || !sGk) {
    free(Ik);
    free(sk);
    free(Gk);
    free(sGk);
    return OR_ENOMEM;
  }
  for (int k = 0; k < itmx && !st; ++k) {
    uint32_t it = (uint32_t)(*iteration);
    st = iteration_sums(id, ndim, nbins, edges, prm, nparams, seed, it, batch,
                        ncall, nch, 0, 0, 0.0, 0.0, sums, NULL);
    if (st) break;
    *iteration += 1;
    mean_sigma(sums[0], sums[1], ncall, &Ik[k], &sk[k]);
    for (int p = 0; p < ORACLE_NGRAD; ++p)
      mean_sigma(sums[2 + 2 * p], sums[3 + 2 * p], ncall,
                 &Gk[k * ORACLE_NGRAD + p], &sGk[k * ORACLE_NGRAD + p]);
    if (per_iter) {
      per_iter[2 * k] = Ik[k];
      per_iter[2 * k + 1] = sk[k];
    }
    if (per_iter_grad)
      for (int p = 0; p < ORACLE_NGRAD; ++p) {
        per_iter_grad[(k * ORACLE_NGRAD + p) * 2] = Gk[k * ORACLE_NGRAD + p];
        per_iter_grad[(k * ORACLE_NGRAD + p) * 2 + 1] = sGk[k * ORACLE_NGRAD + p];
      }
  }
  if (!st) {
    double chi2;
    oracle_combine(itmx, Ik, sk, integral, error, &chi2);
    int nzero = 0;
    for (int k = 0; k < itmx; ++k) nzero += !(sk[k] > 0.0);
    for (int p = 0; p < ORACLE_NGRAD; ++p) {
      double num = 0.0, den = 0.0, var = 0.0;
      for (int k = 0; k < itmx; ++k) {
        double wt;
        if (nzero > 0)
          wt = (sk[k] > 0.0) ? 0.0 : 1.0;
        else
          wt = 1.0 / (sk[k] * sk[k]);
        num += wt * Gk[k * ORACLE_NGRAD + p];
        den += wt;
        var += wt * wt * sGk[k * ORACLE_NGRAD + p] * sGk[k * ORACLE_NGRAD + p];
      }
      grad[p] = num / den;
      grad_err[p] = sqrt(var) / den;
    }
  }
  free(Ik);
  free(sk);
  free(Gk);
  free(sGk);
  return st;
}

/* ------------------------------------------------------------------------
 * VEGAS+: adaptive stratified sampling on top of the VEGAS map (Lepage,
 * J. Comput. Phys. 439 (2021) 110386, a later form of the method the paper
 * cites in Section 2.1).  As restated here:
 *   - the unit cube of the map's input y is cut into NH = s^d hypercubes,
 *     s the largest integer with 4 s^d <= C and s^d <= ORACLE_PLUS_MAX_CUBES
 *     (so at least 4 events per hypercube on average); hypercube h has
 *     coordinates c_a = floor(h / s^a) mod s and volume 1/NH;
 *   - hypercube h gets n_h >= 2 events (uniform floor(C/NH) at the start);
 *     events are numbered hypercube by hypercube, so event e lies in the h
 *     with o_h <= e < o_h + n_h (o the running sum of n);
 *   - event e's word on axis a is the stratified word
 *     r' = floor((c_a 2^32 + r_a) / s), y = r'/2^32 in [c_a/s, (c_a+1)/s),
 *     with r_a its Philox word; then the VEGAS map as before: F = J g(x);
 *   - per hypercube, the sample mean and variance of F (sequential sums in
 *     event order): m_h = S1h/n_h, v_h = (S2h - S1h^2/n_h)/(n_h - 1) (>= 0);
 *   - I_k = sum_h m_h/NH (as sum_e F a_h / C, a_h = C/(NH n_h)), and
 *     sigma_k^2 = sum_h v_h/n_h / NH^2;
 *   - the map is trained on d_{a,i} = sum over the events in bin i of axis a
 *     of q^2, q = F b_h, b_h = sqrt(1/(NH n_h)): an estimate of the integral
 *     of F^2 over the slab (each event stands for the volume 1/(NH n_h));
 *   - the next allocation: d_h = v_h^(beta/2), n_h = max(2, floor(C d_h/D)),
 *     D = sum_h d_h (uniform again if D = 0), with the damping
 *     beta in {0, 1/4, 1/2, 3/4, 1}; v^(beta/2) is formed in FP32 from
 *     correctly rounded operations only (three square roots and products)
 *     after an exact split of v's exponent, so that the decision can be
 *     reproduced exactly anywhere.
 * ---------------------------------------------------------------------- */
#define ORACLE_PLUS_MAX_CUBES (1 << 22)

int oracle_plus_nstrat(int ndim, int64_t ncall) {
  if (ndim < 1 || ncall < 8) return 1;
  int64_t s = 1;
  for (;;) {
    int64_t t = s + 1, p = 1;
    int over = 0;
    for (int a = 0; a < ndim; ++a) {
      p *= t;
      if (p > ORACLE_PLUS_MAX_CUBES || 4 * p > ncall) {
        over = 1;
        break;
      }
    }
    if (over) return (int)s;
    s = t;
  }
}

uint32_t oracle_plus_word(uint32_t r, uint32_t c, uint32_t s) {
  return (uint32_t)((((uint64_t)c << 32) | (uint64_t)r) / (uint64_t)s);
}

/* v^(j/8) for v >= 0 finite (j = 4 beta): v = t 2^(8q), t in [1/2, 128),
 * t rounded to FP32, y = sqrt(sqrt(sqrt(t))) in FP32, y^j by FP32 products,
 * times 2^(q j) exactly. */
double oracle_plus_weight(double v, int j) {
  if (j == 0) return 1.0;
  if (!(v > 0.0)) return 0.0;
  int e;
  double m = frexp(v, &e); /* v = m 2^e, m in [1/2, 1) */
  int q = e >= 0 ? e / 8 : -((-e + 7) / 8);
  int r = e - 8 * q; /* 0 <= r < 8 */
  volatile float t = (float)ldexp(m, r);
  volatile float y = sqrtf(sqrtf(sqrtf(t)));
  volatile float p = y;
  for (int k = 1; k < j; ++k) p = p * y;
  return ldexp((double)p, q * j);
}

/* Allocation of the next iteration from the hypercubes' variances. */
int oracle_plus_allocate(int64_t nh, int64_t ncall, int beta_j, const double* var,
                         int32_t* n) {
  if (nh < 1 || ncall < 2 * nh || beta_j < 0 || beta_j > 4) return OR_EINVAL;
  double* d = (double*)malloc(sizeof(double) * (size_t)nh);
  if (!d) return OR_ENOMEM;
  csum_t D = {0.0, 0.0};
  for (int64_t h = 0; h < nh; ++h) {
    d[h] = oracle_plus_weight(var[h], beta_j);
    csum_add(&D, d[h]);
  }
  double Dv = csum_value(&D);
  for (int64_t h = 0; h < nh; ++h) {
    int64_t k;
    if (Dv > 0.0) {
      double x = (double)ncall * d[h] / Dv;
      k = (int64_t)floor(x);
    } else {
      k = ncall / nh;
    }
    n[h] = (int32_t)(k > 2 ? k : 2);
  }
  free(d);
  return OR_OK;
}

/* itmx VEGAS+ iterations (one stage).  alloc (NH counts, in/out): the
 * allocation of the first iteration (alloc[0] <= 0: uniform), on return the
 * allocation for the next one.  nstrat: strata per axis (0: as above).
 * calls (nullable): the events of each iteration.  last_sums (nullable):
 * (sum w, sum w^2, d[ndim*nbins]) of the last iteration with w = F a_h;
 * last_var, last_mean (nullable): its per-hypercube variances v_h and means
 * m_h.  With adapt = 0 the grid and the allocation stay as they are. */
int oracle_iterate_plus(int ndim, int nbins, uint64_t seed, uint32_t batch,
                        uint64_t* iteration, int64_t ncall, int itmx, int id,
                        const double* prm, int nparams, double alpha, int adapt,
                        int beta_j, int nstrat, double* edges, int32_t* alloc,
                        double* integral, double* error, double* chi2dof,
                        double* per_iter, int64_t* calls, double* last_sums,
                        double* last_var, double* last_mean, int64_t* nonfinite) {
  if (ndim < 1 || ndim > ORACLE_MAX_DIM || nbins < 2 || ncall < 8 ||
      ncall > ((int64_t)1 << 30) || itmx < 1 || beta_j < 0 || beta_j > 4)
    return OR_EINVAL;
  int st = check_integrand(id, ndim, nparams);
  if (st) return st;
  const int s = nstrat > 0 ? nstrat : oracle_plus_nstrat(ndim, ncall);
  int64_t NH = 1;
  for (int a = 0; a < ndim; ++a) NH *= s;
  if (NH > ORACLE_PLUS_MAX_CUBES || 4 * NH > ncall) return OR_EINVAL;
  if (alloc[0] <= 0)
    for (int64_t h = 0; h < NH; ++h) alloc[h] = (int32_t)(ncall / NH);
  const int nd = 2 + ndim * nbins;
  const double C = (double)ncall;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(NH + 1));
  double* var = (double*)malloc(sizeof(double) * (size_t)NH);
  double* mean = (double*)malloc(sizeof(double) * (size_t)NH);
  double* Ik = (double*)malloc(sizeof(double) * itmx);
  double* sk = (double*)malloc(sizeof(double) * itmx);
  double* sums = (double*)malloc(sizeof(double) * nd);
  if (!off || !var || !mean || !Ik || !sk || !sums) {
    free(off);
    free(var);
    free(mean);
    free(Ik);
    free(sk);
    free(sums);
    return OR_ENOMEM;
  }
  int64_t bad_all = 0;
  for (int k = 0; k < itmx && !st; ++k) {
    const uint32_t it = (uint32_t)(*iteration);
    off[0] = 0;
    for (int64_t h = 0; h < NH; ++h) off[h + 1] = off[h] + alloc[h];
    const int64_t Cp = off[NH];
    double* F = (double*)malloc(sizeof(double) * (size_t)(Cp > 0 ? Cp : 1));
    csum_t* total = (csum_t*)calloc((size_t)nd, sizeof(csum_t));
    if (!F || !total) {
      free(F);
      free(total);
      st = OR_ENOMEM;
      break;
    }
    const int64_t nchunks = (Cp + ORACLE_CHUNK - 1) / ORACLE_CHUNK;
    int64_t bad_it = 0;
    int fail = 0;
#pragma omp parallel
    {
      csum_t* part = (csum_t*)malloc(sizeof(csum_t) * (size_t)nd);
      if (!part) {
#pragma omp atomic write
        fail = 1;
      }
#pragma omp for ordered schedule(static, 1)
      for (int64_t ch = 0; ch < nchunks; ++ch) {
        int64_t bad = 0;
        if (part) {
          memset(part, 0, sizeof(csum_t) * (size_t)nd);
          const int64_t e0 = ch * ORACLE_CHUNK;
          const int64_t e1 = e0 + ORACLE_CHUNK < Cp ? e0 + ORACLE_CHUNK : Cp;
          /* the hypercube of e0: the last h with off[h] <= e0 */
          int64_t lo = 0, hi = NH;
          while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (off[mid] <= e0)
              lo = mid;
            else
              hi = mid;
          }
          int64_t h = lo;
          for (int64_t ev = e0; ev < e1; ++ev) {
            while (ev >= off[h + 1]) ++h;
            uint32_t words[ORACLE_MAX_DIM];
            double x[ORACLE_MAX_DIM];
            int32_t bins[ORACLE_MAX_DIM];
            oracle_event_words(seed, it, batch, (uint64_t)ev, ndim, words);
            int64_t rest = h;
            double J = 1.0;
            for (int a = 0; a < ndim; ++a) {
              uint32_t c = (uint32_t)(rest % s);
              rest /= s;
              uint32_t rw = oracle_plus_word(words[a], c, (uint32_t)s);
              double xa;
              J *= oracle_grid_map(edges + (size_t)a * (nbins + 1), nbins, rw, &xa);
              x[a] = xa;
              int32_t bi;
              double fr;
              oracle_bin_map(rw, nbins, &bi, &fr);
              bins[a] = bi;
            }
            double Fe = J * integrand_point(id, ndim, x, prm, nparams, NULL, NULL);
            if (!isfinite(Fe)) {
              ++bad;
              F[ev] = 0.0;
              continue;
            }
            F[ev] = Fe;
            const double nhd = (double)NH * (double)alloc[h];
            const double ah = C / nhd, bh = sqrt(1.0 / nhd);
            const double w = Fe * ah, q = Fe * bh;
            csum_add(&part[0], w);
            csum_add(&part[1], w * w);
            for (int a = 0; a < ndim; ++a) csum_add(&part[2 + a * nbins + bins[a]], q * q);
          }
        }
#pragma omp ordered
        {
          if (part)
            for (int j = 0; j < nd; ++j) csum_add(&total[j], csum_value(&part[j]));
          bad_it += bad;
        }
      }
      free(part);
    }
    if (fail) {
      free(F);
      free(total);
      st = OR_ENOMEM;
      break;
    }
    for (int j = 0; j < nd; ++j) sums[j] = csum_value(&total[j]);
    free(total);
    /* per hypercube: sequential sums over its events in order */
#pragma omp parallel for schedule(static)
    for (int64_t h = 0; h < NH; ++h) {
      double s1 = 0.0, s2 = 0.0;
      for (int64_t ev = off[h]; ev < off[h + 1]; ++ev) {
        s1 += F[ev];
        s2 += F[ev] * F[ev];
      }
      const double n = (double)alloc[h];
      double v = (s2 - s1 * s1 / n) / (n - 1.0);
      var[h] = v > 0.0 ? v : 0.0;
      mean[h] = s1 / n;
    }
    free(F);
    csum_t V = {0.0, 0.0};
    for (int64_t h = 0; h < NH; ++h) csum_add(&V, var[h] / (double)alloc[h]);
    const double var_k = csum_value(&V) / ((double)NH * (double)NH);
    Ik[k] = sums[0] / C;
    sk[k] = var_k > 0.0 ? sqrt(var_k) : 0.0;
    if (per_iter) {
      per_iter[2 * k] = Ik[k];
      per_iter[2 * k + 1] = sk[k];
    }
    if (calls) calls[k] = Cp;
    bad_all += bad_it;
    *iteration += 1;
    if (k == itmx - 1) {
      if (last_sums) memcpy(last_sums, sums, sizeof(double) * nd);
      if (last_var) memcpy(last_var, var, sizeof(double) * (size_t)NH);
      if (last_mean) memcpy(last_mean, mean, sizeof(double) * (size_t)NH);
    }
    if (adapt) {
      oracle_refine(ndim, nbins, alpha, sums + 2, edges);
      st = oracle_plus_allocate(NH, ncall, beta_j, var, alloc);
    }
  }
  if (!st) oracle_combine(itmx, Ik, sk, integral, error, chi2dof);
  if (nonfinite) *nonfinite = bad_all;
  free(off);
  free(var);
  free(mean);
  free(Ik);
  free(sk);
  free(sums);
  return st;
}
