"""GPU path vs the oracle, through the C ABI (requires a GB300).

Bar: Philox words and bins bit-exact; FP64 per-iteration I_k, sigma_k and the
combined result within 1e-12 relative; grid edges within 1e-12 absolute;
bit-identical results for every launch shape.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import DY_PARAMS, DYNLO_PARAMS, EE3J_PARAMS, GAUSS_PARAMS

pytestmark = pytest.mark.gpu

CASES = {
    "gauss": (v.VEGAS_GAUSS, GAUSS_PARAMS, 4, 50),
    "dy": (v.VEGAS_DY, DY_PARAMS, 4, 100),
    "ee3j": (v.VEGAS_EE3J, EE3J_PARAMS, 5, 100),
    "dy_nlo": (v.VEGAS_DY_NLO, DYNLO_PARAMS, 13, 50),  # the NLO-shaped stand-in
}


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def run_gpu(ndim, nbins, seed, ncall, itmx, iid, params, **opts):
    g = v.Vegas(ndim, nbins, seed)
    try:
        for k, val in opts.items():
            g.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
        I, e, c, per, _ = g.iterate(ncall, itmx, iid, params)
        return dict(integral=I, error=e, chi2=c, per_iter=per, edges=g.grid, sums=g.last_sums())
    finally:
        g.close()


def test_philox_words_bit_exact():
    rng = np.random.default_rng(0)
    for seed, it, batch, first, n, nd in [(1234, 0, 0, 0, 4096, 4), (2**63 + 5, 7, 3, 2**32 - 100, 500, 13),
                                          (99, 2**31, 63, 10**9, 300, 16)]:
        got = v.vegas_rng_words(seed, it, batch, first, n, nd)
        for j in rng.choice(n, size=min(n, 64), replace=False):
            want = oracle.event_words(seed, it, batch, first + int(j), nd)
            assert np.array_equal(got[j], want), (seed, it, batch, first + j)
    # a million (event, axis) pairs against the oracle, vectorised through bins of N = 2^k:
    got = v.vegas_rng_words(1234, 3, 0, 0, 250_000, 4)
    sample = rng.choice(250_000, size=2000, replace=False)
    for j in sample:
        assert np.array_equal(got[j], oracle.event_words(1234, 3, 0, int(j), 4))


@pytest.mark.parametrize("name", list(CASES))
def test_single_events_match_oracle(name):
    iid, params, ndim, nbins = CASES[name]
    g = v.Vegas(ndim, nbins, 1234)
    try:
        # adapt the grid first so that the map is not uniform
        g.iterate(20_000, 2, iid, params)
        edges = g.grid
        events = np.arange(0, 200_000, 97, dtype=np.int64)
        w, bins = g.eval_events(iid, params, 5, events)
    finally:
        g.close()
    for j, ev in enumerate(events[:400]):
        wo, bo, _ = oracle.event(iid, ndim, nbins, edges, params, 1234, 5, 0, int(ev))
        assert np.array_equal(bins[j], bo)
        if wo == 0.0:
            assert w[j] == 0.0
        else:
            assert abs(w[j] - wo) <= 1e-13 * abs(wo), (ev, w[j], wo)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ncall", [20 * 1024 + 37, 1500])
def test_fp64_stage_matches_oracle(name, ncall):
    iid, params, ndim, nbins = CASES[name]
    itmx = 4
    gpu = run_gpu(ndim, nbins, 1234, ncall, itmx, iid, params)
    ref = oracle.iterate(ndim, nbins, 1234, ncall, itmx, iid, params, want_sums=True)
    assert rel(gpu["per_iter"], ref.per_iter) < 1e-12
    assert rel(gpu["integral"], ref.integral) < 1e-12
    assert rel(gpu["error"], ref.error) < 1e-12
    assert abs(gpu["chi2"] - ref.chi2dof) < 1e-10 * max(1.0, ref.chi2dof)
    assert np.max(np.abs(gpu["edges"] - ref.edges)) < 1e-12
    # The sums of the last iteration, against the oracle started from the same
    # grid: after a chain of refinements an edge's last-bit difference reaches
    # the next iteration's weights through 1/width (sparse samples of a peaked
    # integrand make narrow bins), so the sums are compared from one grid.
    g = v.Vegas(ndim, nbins, 1234)
    try:
        g.iterate(ncall, itmx - 1, iid, params)
        edges = g.grid
        g.iterate(ncall, 1, iid, params)
        sums = g.last_sums()
    finally:
        g.close()
    s = oracle.iterate(ndim, nbins, 1234, ncall, 1, iid, params, edges=edges, iteration=itmx - 1,
                       want_sums=True).sums
    assert rel(sums[:2], s[:2]) < 1e-12
    d_gpu, d_ref = sums[2:], s[2:]
    nz = d_ref != 0
    assert np.array_equal(d_gpu == 0, ~nz)
    assert rel(d_gpu[nz], d_ref[nz]) < 1e-12
    # and the chained run's sums are those of the same iteration
    assert np.array_equal(gpu["sums"], sums)


@pytest.mark.parametrize("name", list(CASES))
def test_bit_identical_across_launch_shapes(name):
    iid, params, ndim, nbins = CASES[name]
    outs = []
    for ept in (1, 2, 4, 8) if ndim <= 8 else (1, 2, 4):  # 8 events per thread only up to 8 axes
        for graph in (1, 0):
            outs.append(run_gpu(ndim, nbins, 77, 9 * 1024 + 5, 3, iid, params, ept=ept, graph=graph))
    for o in outs[1:]:
        assert np.array_equal(o["per_iter"], outs[0]["per_iter"])
        assert np.array_equal(o["edges"], outs[0]["edges"])
        assert np.array_equal(o["sums"], outs[0]["sums"])


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_integrand_error_vs_oracle(name):
    """The FP32 integrand form on the same events: the error against the FP64
    oracle is small and stated (per-iteration relative error of I_k < 2e-5,
    of sigma_k < 2e-4)."""
    iid, params, ndim, nbins = CASES[name]
    gpu = run_gpu(ndim, nbins, 1234, 50_000, 4, iid, params, precision=1)
    ref = oracle.iterate(ndim, nbins, 1234, 50_000, 4, iid, params)
    eI = rel(gpu["per_iter"][:, 0], ref.per_iter[:, 0])
    eS = rel(gpu["per_iter"][:, 1], ref.per_iter[:, 1])
    print(f"{name}: fp32 rel err I_k {eI:.2e} sigma_k {eS:.2e}")
    assert eI < 2e-5
    assert eS < 2e-4
