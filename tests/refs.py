"""Independent reference values for pinning the oracle.

Everything here is derived from textbook physics or mathematics by a route
other than the oracle's: helicity amplitudes instead of the (A, B) form of
the Drell-Yan cross section, adaptive quadrature in the physical variables
(tau, y) instead of VEGAS over the unit cube, closed forms via erf and the
dilogarithm.  Nothing here calls the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

GEV2_TO_PB = 0.3893794e9
NC = 3.0
UP = (2.0 / 3.0, 0.5)
DOWN = (-1.0 / 3.0, -0.5)
MUON = (-1.0, -0.5)
FLAVOURS = (UP, DOWN, DOWN, UP, DOWN)  # u d s c b


def gauss_exact(ndim: int, sigma: float = 0.1) -> float:
    """prod_a int_0^1 exp(-(x-1/2)^2/(2 sigma^2)) dx = (sigma sqrt(2 pi) erf(1/(2 sqrt2 sigma)))^d."""
    one = sigma * math.sqrt(2 * math.pi) * math.erf(0.5 / (sigma * math.sqrt(2)))
    return one ** ndim


def ee3j_exact(y: float) -> float:
    """Integral of (x1^2+x2^2)/((1-x1)(1-x2)) over the region y_ij > y
    (massless 3-parton phase space, unit normalisation), in closed form.
    Li2(z) = scipy.special.spence(1 - z)."""
    li2 = special.spence(1.0 - y / (1.0 - y))
    return ((3 - 6 * y) * math.log(y / (1 - 2 * y)) + 2 * math.log(y / (1 - y)) ** 2
            + 2.5 - 6 * y - 4.5 * y * y + 4 * li2 - math.pi ** 2 / 3)


def ee3j_quadrature(y: float) -> float:
    f = lambda x2, x1: (x1 * x1 + x2 * x2) / ((1 - x1) * (1 - x2))
    # x1 in (2y, 1-y); x2 in (1+y-x1, 1-y)
    val, _ = integrate.dblquad(f, 2 * y, 1 - y, lambda x1: 1 + y - x1, lambda x1: 1 - y,
                               epsabs=0, epsrel=1e-12)
    return val


def _helicity_F(fq, shat, MZ, GZ, sw2):
    """F_ij = Q_q Q_l + g_i^q g_j^l / (sw2 cw2) * shat / (shat - M^2 + i Gamma M),
    i = quark chirality, j = lepton chirality; g_L = T3 - Q sw2, g_R = -Q sw2."""
    Qq, T3q = fq
    Ql, T3l = MUON
    cw2 = 1.0 - sw2
    prop = shat / complex(shat - MZ * MZ, GZ * MZ)
    gq = {"L": T3q - Qq * sw2, "R": -Qq * sw2}
    gl = {"L": T3l - Ql * sw2, "R": -Ql * sw2}
    return {i + j: Qq * Ql + gq[i] * gl[j] / (sw2 * cw2) * prop for i in "LR" for j in "LR"}


def dy_dsigma_domega_helicity(fq, shat, c, MZ, GZ, sw2, alpha):
    """q qbar -> mu- mu+ in helicity amplitudes; c = cos(quark, mu-).  Same
    chiralities go with (1+c)^2, opposite ones with (1-c)^2."""
    F = _helicity_F(fq, shat, MZ, GZ, sw2)
    same = abs(F["LL"]) ** 2 + abs(F["RR"]) ** 2
    opp = abs(F["LR"]) ** 2 + abs(F["RL"]) ** 2
    return alpha ** 2 / (16 * shat * NC) * (same * (1 + c) ** 2 + opp * (1 - c) ** 2)


def dy_sigma_hat(fq, shat, MZ, GZ, sw2, alpha):
    """Angle-integrated: int dOmega (1 +- c)^2 = 16 pi / 3."""
    F = _helicity_F(fq, shat, MZ, GZ, sw2)
    return math.pi * alpha ** 2 / (3 * shat * NC) * sum(abs(v) ** 2 for v in F.values())


def dy_sigma_quadrature(params, epsrel=1e-10, m_range=None) -> float:
    """sigma(pp -> mu+ mu-) in pb by adaptive quadrature over (m_mumu, y):
    sum_q int dtau dy [f_q(x1) f_qbar(x2) + f_qbar(x1) f_q(x2)] sigmahat_q(tau s).
    m_range = (m_a, m_b) restricts the dilepton mass to that interval (inside
    the generated range): the cross section in one bin of m_mumu."""
    sqrt_s, MZ, GZ, sw2, alpha, mlo, mhi, a, b, N = params
    if m_range is not None:
        mlo, mhi = max(mlo, m_range[0]), min(mhi, m_range[1])
        if not mhi > mlo:
            return 0.0
    s = sqrt_s ** 2
    fq = lambda x: N * x ** a * (1 - x) ** b
    fqb = lambda x: 0.2 * N * x ** a * (1 - x) ** (b + 4)

    def inner(m):
        tau = m * m / s
        shat = tau * s
        sig = sum(dy_sigma_hat(f, shat, MZ, GZ, sw2, alpha) for f in FLAVOURS)
        Y = -0.5 * math.log(tau)
        rt = math.sqrt(tau)

        def lumi(y):
            x1, x2 = rt * math.exp(y), rt * math.exp(-y)
            return fq(x1) * fqb(x2) + fqb(x1) * fq(x2)

        L, _ = integrate.quad(lumi, -Y, Y, epsabs=0, epsrel=epsrel * 0.1, limit=200)
        return L * sig * 2 * m / s  # dtau = 2 m dm / s

    pts = [MZ] if mlo < MZ < mhi else None
    val, _ = integrate.quad(inner, mlo, mhi, points=pts, epsabs=0, epsrel=epsrel, limit=400)
    return val * GEV2_TO_PB


def gauss_bin(a: float, b: float, ndim: int, sigma: float = 0.1) -> float:
    """Integral of the product Gaussian over x_0 in [a, b] (inside [0, 1]) and
    the other axes over [0, 1], via erf."""
    r = sigma * math.sqrt(2.0)
    a, b = max(a, 0.0), min(b, 1.0)
    if not b > a:
        return 0.0
    first = sigma * math.sqrt(math.pi / 2) * (math.erf((b - 0.5) / r) - math.erf((a - 0.5) / r))
    return first * gauss_exact(ndim - 1, sigma)


def ee3j_thrust_density(T: float) -> float:
    """d sigma / dT of (x1^2+x2^2)/((1-x1)(1-x2)) over the massless 3-parton
    phase space (unit normalisation), T = max(x1, x2, x3) in (2/3, 1): the
    classic leading-order thrust distribution (De Rujula, Ellis, Floratos,
    Gaillard 1978)."""
    return (2.0 * (3 * T * T - 3 * T + 2) / (T * (1 - T)) * math.log((2 * T - 1) / (1 - T))
            - 3.0 * (3 * T - 2) * (2 - T) / (1 - T))


def ee3j_thrust_bin(a: float, b: float, y: float) -> float:
    """Integral of the thrust distribution over [a, b] intersected with the
    region the cut y_ij > y leaves, 2/3 < T < 1 - y (for three massless
    partons y_ij = 1 - x_k, so the cut is exactly T < 1 - y)."""
    a, b = max(a, 2.0 / 3.0), min(b, 1.0 - y)
    if not b > a:
        return 0.0
    val, _ = integrate.quad(ee3j_thrust_density, a, b, epsabs=0, epsrel=1e-12, limit=200)
    return val


def pulls(values, errors, exact):
    v = np.asarray(values)
    e = np.asarray(errors)
    return (v - exact) / e
