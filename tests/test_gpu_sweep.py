"""A seeded sweep of random configurations against the oracle (FP64 form):
integrand, 1-16 axes, 2-1024 bins, ragged call counts, Philox batch words.
Each iteration is compared from the same grid (the oracle restarted from the
GPU's grid and counter) at 1e-12, and so is the grid it refines to.

sigma_k^2 = (S2/C - I_k^2)/(C-1) cancels when the weights are nearly equal:
a relative error eps in S2 becomes kappa eps in sigma_k^2, kappa =
(S2/C) / (S2/C - I_k^2).  The GPU's S2 is exact, rounded once; the oracle's
compensated S2 carries about an ulp.  So sigma_k is held to 1e-12 plus
8 eps kappa (the shifted Gaussian's nearly constant weights give kappa ~ 1e4)."""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import (DY_PARAMS, DYNLO_PARAMS, EE3J_PARAMS, GAUSS_PARAMS,
                                              GAUSS_SHIFTED_PARAMS)

pytestmark = pytest.mark.gpu

_RNG = np.random.default_rng(20260)
_INTEGRANDS = [(v.VEGAS_GAUSS, GAUSS_PARAMS, 1), (v.VEGAS_GAUSS, GAUSS_SHIFTED_PARAMS, 1),
               (v.VEGAS_DY, DY_PARAMS, 4), (v.VEGAS_EE3J, EE3J_PARAMS, 5),
               (v.VEGAS_DY_NLO, DYNLO_PARAMS, 4)]


def _configs(n=24):
    out = []
    for i in range(n):
        iid, params, dmin = _INTEGRANDS[i % len(_INTEGRANDS)]
        ndim = int(_RNG.integers(dmin, 17))
        nbins = int(_RNG.choice([2, 3, 17, 50, 100, 255, 1024]))
        while ndim * nbins > 4096:
            nbins //= 2
        nbins = max(nbins, 2)
        ncall = int(_RNG.integers(2, 40_000))
        batch = int(_RNG.integers(0, 1 << 10))
        out.append((iid, params, ndim, nbins, ncall, batch))
    return out


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


@pytest.mark.parametrize("iid,params,ndim,nbins,ncall,batch", _configs())
def test_random_configuration_matches_oracle(iid, params, ndim, nbins, ncall, batch):
    g = v.Vegas(ndim, nbins, 4242)
    try:
        g.set(v.VEGAS_OPT_BATCH_ID, batch)
        for k in range(2):
            edges = g.grid
            I, e, c, per, st = g.iterate(ncall, 1, iid, params, allow_nonfinite=True)
            ref = oracle.iterate(ndim, nbins, 4242, ncall, 1, iid, params, edges=edges,
                                 iteration=k, batch=batch)
            assert rel(per[:, 0], ref.per_iter[:, 0]) < 1e-12, (k, per, ref.per_iter)
            s = ref.per_iter[0, 1]
            I = ref.per_iter[0, 0]
            var_c = s * s * (ncall - 1)  # S2/C - I^2
            kappa = (var_c + I * I) / var_c if var_c > 0 else 1.0
            tol = 1e-12 + 8 * np.finfo(float).eps * kappa
            assert abs(per[0, 1] - s) <= tol * s, (k, per, ref.per_iter, kappa)
            assert np.max(np.abs(g.grid - ref.edges)) < 1e-12, k
    finally:
        g.close()
