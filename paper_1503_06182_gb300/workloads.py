"""Seeded synthetic workloads (shared by the tests, the oracle checks and the bench).

This module holds the workload *descriptions* only -- dimensions, call counts,
integrand ids and physics parameters, plus a seeded generator for the batched
workload.  It contains none of the VEGAS arithmetic, so the oracle and the
CUDA path can both draw their inputs from it without sharing any of the
method.

The paper's benchmark process (Section 3.2: PP -> H(-> b bbar) + 2 jets, a
10-dimensional LO and a 13-dimensional NLO integral, run as 4 x 1,000 warm-up
plus 10 x 10,000 production VEGAS events) needs MCFM's matrix elements and
parton-density sets, which are not available.  The workloads below stand in
for it with integrands whose integrals are known in closed form or by
quadrature, at the dimensions and call counts the paper's runs use.
"""
from __future__ import annotations

from dataclasses import dataclass, field

GAUSS, DY, EE3J, DYNLO = 0, 1, 2, 3
INTEGRAND_NAMES = {GAUSS: "gauss", DY: "drell_yan", EE3J: "ee_qqg", DYNLO: "drell_yan_nlo_shaped"}

# LO pp -> gamma*/Z -> mu+ mu- at sqrt(s) = 14 TeV:
# (sqrt_s, M_Z, Gamma_Z, sin^2 theta_W, alpha, m_lo, m_hi, a, b, N)
DY_PARAMS = (14000.0, 91.1876, 2.4952, 0.2312, 1.0 / 128.0, 60.0, 120.0, -0.5, 3.0, 1.0)
# indices of (M_Z, Gamma_Z, sin^2 theta_W, a, b) inside DY_PARAMS
DY_GRAD_INDEX = (1, 2, 3, 7, 8)
GAUSS_PARAMS = (0.1,)
# the Gaussian minus a constant 0.1: negative weights over most of the cube
# (as subtraction terms give at NLO), a negative integral in d = 2
GAUSS_SHIFTED_PARAMS = (0.1, 0.1)
# NLO-shaped stand-in: the Drell-Yan parameters, then beta of the extra axes'
# factors exp(beta cos 2 pi x) / I0(beta)
DYNLO_PARAMS = DY_PARAMS + (0.5,)
EE3J_PARAMS = (0.01, 91.1876)

SEED = 1234


@dataclass(frozen=True)
class Workload:
    name: str
    integrand: int
    ndim: int
    nbins: int
    ncall: int
    itmx: int
    params: tuple
    precision: str = "fp64"  # "fp64" or "fp32" (integrand arithmetic)
    seed: int = SEED
    alpha: float = 1.5
    extra: dict = field(default_factory=dict)


# The five configurations of the build (shapes of the paper-style workloads).
CONFIGS = {
    "gauss4": Workload("gauss4", GAUSS, 4, 50, 100_000, 5, GAUSS_PARAMS, "fp64"),
    "dy": Workload("dy", DY, 4, 100, 1_000_000, 10, DY_PARAMS, "fp32"),
    "ee3j": Workload("ee3j", EE3J, 5, 100, 10_000_000, 10, EE3J_PARAMS, "fp32"),
    "dy_grad": Workload("dy_grad", DY, 4, 100, 100_000_000, 10, DY_PARAMS, "fp32"),
    "batch64": Workload("batch64", -1, 0, 100, 0, 10, (), "fp32"),
}

# Paper-shaped extra: 4 x 1,000 warm-up + 10 x 10,000 production events in
# 10 and 13 dimensions (Section 3.2).
PAPER_SHAPED = {
    "gauss10_paper": dict(ndim=10, warmup=(1000, 4), production=(10_000, 10)),
    "gauss13_paper": dict(ndim=13, warmup=(1000, 4), production=(10_000, 10)),
}


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): a tiny seeded generator for the
    batched workload's specification.  It is not the event generator."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.next_u64() % (hi - lo + 1)


@dataclass(frozen=True)
class BatchMember:
    index: int
    integrand: int
    ndim: int
    ncall: int
    params: tuple


def batch_spec(n: int = 64, seed: int = SEED, ncall_lo: float = 1e4, ncall_hi: float = 1e7,
               ndim_lo: int = 2, ndim_hi: int = 12) -> list[BatchMember]:
    """The batched workload: n independent integrations.

    ndim is uniform in [ndim_lo, ndim_hi]; the Drell-Yan and 3-jet forms need
    at least 4 and 5 axes, so they use max(ndim, 4) and max(ndim, 5) (the
    extra axes are flat); calls per iteration are log-uniform in
    [ncall_lo, ncall_hi]; the integrand is chosen uniformly among the three
    forms; Drell-Yan draws M_Z in [80, 100] GeV and the 3-jet form y_cut in
    [0.005, 0.05]."""
    import math

    rng = SplitMix64(seed)
    out = []
    for i in range(n):
        kind = rng.randint(0, 2)
        ndim = rng.randint(ndim_lo, ndim_hi)
        u = rng.uniform()
        ncall = int(round(math.exp(math.log(ncall_lo) + u * (math.log(ncall_hi) - math.log(ncall_lo)))))
        v = rng.uniform()
        if kind == GAUSS:
            params = GAUSS_PARAMS
        elif kind == DY:
            ndim = max(ndim, 4)
            p = list(DY_PARAMS)
            p[1] = 80.0 + 20.0 * v
            params = tuple(p)
        else:
            ndim = max(ndim, 5)
            params = (0.005 + 0.045 * v, EE3J_PARAMS[1])
        out.append(BatchMember(i, kind, ndim, ncall, params))
    return out
