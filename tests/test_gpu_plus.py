"""GPU VEGAS+ (adaptive stratified sampling) against the oracle, through the C ABI.

Each iteration is compared from the same state (grid, allocation, iteration
counter): the estimate to 1e-12, the refined grid to 1e-12, the
per-hypercube variances to 1e-11 plus 1e-13 of their scale (the variance
formula cancels where a hypercube's values are nearly equal), and the error
sigma_k to the bound those variances' tolerance puts on it.  The next
allocation is the oracle's allocation rule applied to the GPU's own
variances, exactly; against the oracle's own allocation it differs by at most
one event in few hypercubes (those whose weights the small variance
differences move across a floor).  The GPU itself is bit-identical for every
launch shape.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import (DY_PARAMS, DYNLO_PARAMS, EE3J_PARAMS, GAUSS_PARAMS,
                                              GAUSS_SHIFTED_PARAMS)

pytestmark = pytest.mark.gpu

CASES = {
    "gauss_d2": (v.VEGAS_GAUSS, GAUSS_PARAMS, 2, 50),
    "gauss_signed_d2": (v.VEGAS_GAUSS, GAUSS_SHIFTED_PARAMS, 2, 40),
    "dy": (v.VEGAS_DY, DY_PARAMS, 4, 100),
    "ee3j": (v.VEGAS_EE3J, EE3J_PARAMS, 5, 60),
    "dy_nlo": (v.VEGAS_DY_NLO, DYNLO_PARAMS, 13, 30),
}


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def var_agrees(got, ref, alloc):
    """Per-hypercube variances: v = (sum F^2 - (sum F)^2/n)/(n-1) cancels where
    a hypercube's values are nearly equal, so the two sides (F equal to
    ~1e-15) agree to 1e-11 of v plus 1e-13 of the scale m^2 n/(n-1)."""
    n = np.asarray(alloc, float)
    scale = ref.mean ** 2 * n / (n - 1)
    assert np.all(np.abs(got - ref.var) <= 1e-11 * ref.var + 1e-13 * scale)


def per_agrees(per, ref, alloc):
    """(I_k, sigma_k) of one iteration: I_k to 1e-12 (exact sums rounded
    once); sigma_k^2 = sum_h v_h/n_h / NH^2 to the sum of the variances' own
    bound (var_agrees) over n_h NH^2.  The GPU adds a hypercube's values in
    4-event segments where the definition adds them one by one, and v_h's
    cancellation turns those few-ulp differences into 1e-11 of sigma_k where
    a hypercube's values are nearly equal (one axis, 262144 strata)."""
    per = np.asarray(per, float).reshape(-1, 2)[-1]
    rp = np.asarray(ref.per_iter, float).reshape(-1, 2)[-1]
    assert abs(per[0] - rp[0]) <= 1e-12 * abs(rp[0])
    n = np.asarray(alloc, float)
    nh = len(n)
    dv = 1e-11 * ref.var + 1e-13 * ref.mean ** 2 * n / (n - 1)
    bound = np.sum(dv / n) / float(nh) ** 2
    assert abs(per[1] ** 2 - rp[1] ** 2) <= bound + 1e-12 * rp[1] ** 2


def gpu_state(iid, params, ndim, nbins, ncall, warm, *, precision="fp64", **opts):
    g = v.Vegas(ndim, nbins, 1234, precision=precision)
    for k, val in opts.items():
        g.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
    g.set(v.VEGAS_OPT_STRAT, 1)
    if warm:
        g.iterate(ncall, warm, iid, params)
    return g


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ncall", [30_000 + 77, 2_000])
def test_plus_iterations_match_oracle(name, ncall):
    iid, params, ndim, nbins = CASES[name]
    g = gpu_state(iid, params, ndim, nbins, ncall, 2)
    try:
        for k in range(2, 5):
            edges = g.grid
            s, alloc, _ = g.strat()
            I, e, c, per, _ = g.iterate(ncall, 1, iid, params)
            s2, alloc2, var = g.strat()
            ref = oracle.iterate_plus(ndim, nbins, 1234, ncall, 1, iid, params, edges=edges,
                                      alloc=alloc, iteration=k)
            assert s == s2 == ref.nstrat
            per_agrees(per, ref, alloc)
            assert np.max(np.abs(g.grid - ref.edges)) < 1e-12, k
            var_agrees(var, ref, alloc)
            # the allocation rule on the GPU's own variances, exactly (the FP32
            # weights are bit-reproducible; only the sum D is formed in
            # another order, 1e-16 apart); the oracle's own allocation
            # differs at most by one event in few hypercubes
            assert np.array_equal(alloc2, oracle.plus_allocate(ncall, var))
            diff = np.abs(alloc2.astype(int) - ref.alloc)
            assert np.max(diff) <= 1 and np.count_nonzero(diff) <= max(3, len(diff) // 200)
            sums = g.last_sums()
            assert rel(sums[:1], ref.sums[:1]) < 1e-12
            dn = ref.sums[2:] != 0
            assert np.array_equal(sums[2:] != 0, dn)
            assert rel(sums[2:][dn], ref.sums[2:][dn]) < 1e-12
    finally:
        g.close()


def test_plus_first_stage_and_combination_match_oracle():
    """A whole stage from the uniform start: the first iteration's allocation
    is uniform on both sides, so the stage's first iteration agrees exactly;
    the stage combination equals the oracle's combination of the GPU's own
    per-iteration records."""
    iid, params, ndim, nbins = CASES["dy"]
    g = gpu_state(iid, params, ndim, nbins, 50_000, 0)
    try:
        I, e, c, per, _ = g.iterate(50_000, 4, iid, params)
    finally:
        g.close()
    ref = oracle.iterate_plus(ndim, nbins, 1234, 50_000, 1, iid, params)
    per_agrees(per[0], ref, np.full(len(ref.var), 50_000 // len(ref.var)))
    Io, eo, co = oracle.combine(per[:, 0], per[:, 1])
    assert rel(I, Io) < 1e-12 and rel(e, eo) < 1e-12 and abs(c - co) < 1e-10 * max(co, 1)


@pytest.mark.parametrize("name", ["dy", "gauss_signed_d2", "dy_nlo"])
def test_plus_bit_identical_across_launch_shapes(name):
    iid, params, ndim, nbins = CASES[name]
    outs = []
    for gr in (1, 0):
        for pd in (1, 0):
            g = gpu_state(iid, params, ndim, nbins, 9 * 1024 + 5, 0, graph=gr, pdl=pd)
            try:
                I, e, c, per, _ = g.iterate(9 * 1024 + 5, 4, iid, params)
                s, alloc, var = g.strat()
                outs.append((per, g.grid, alloc, var, g.last_sums(), np.array([I, e, c])))
            finally:
                g.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_plus_frozen_stage_keeps_allocation():
    iid, params, ndim, nbins = CASES["dy"]
    g = gpu_state(iid, params, ndim, nbins, 20_000, 2)
    try:
        s, a0, _ = g.strat()
        e0 = g.grid
        g.set(v.VEGAS_OPT_ADAPT, 0)
        g.iterate(20_000, 3, iid, params)
        s, a1, _ = g.strat()
        assert np.array_equal(a0, a1) and np.array_equal(e0, g.grid)
    finally:
        g.close()


def test_plus_strat_set_and_validation():
    g = v.Vegas(2, 20, 3)
    try:
        with pytest.raises(v.VegasError):
            g.strat()  # nothing yet
        s = oracle.plus_nstrat(2, 4000)
        nh = s * s
        counts = np.full(nh, 3, np.int32)
        counts[::7] = 9
        g.strat_set(4000, counts)
        s2, got, _ = g.strat()
        assert s2 == s and np.array_equal(got, counts)
        for bad in (np.full(nh, 1, np.int32), np.full(nh, 4000, np.int32), counts[:-1]):
            if len(bad) == nh:
                with pytest.raises(v.VegasError):
                    g.strat_set(4000, bad)
        with pytest.raises(v.VegasError):
            g.strat_set(4, counts)  # below the minimum call count
        # a stage from the set allocation (frozen) equals the oracle's
        g.set(v.VEGAS_OPT_STRAT, 1).set(v.VEGAS_OPT_ADAPT, 0)
        I, e, c, per, _ = g.iterate(4000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)
        ref = oracle.iterate_plus(2, 20, 3, 4000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS, alloc=counts,
                                  adapt=False)
        per_agrees(per, ref, counts)
        with pytest.raises(v.VegasError):  # no histogram with VEGAS+
            g.hist_set(10, 0.0, 1.0)
            g.iterate(4000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)
    finally:
        g.close()


def test_plus_hypercube_across_several_tiles():
    """One hypercube of 2500 events spans four fill tiles (1024 events each),
    beside many 2- and 3-event ones of which some straddle a tile boundary.
    A tile forms the statistics of the hypercubes it holds whole; the others
    come from their segments in every tile they reach, formed once, at the
    first boundary they cross.  sigma_k and the variances agree with the
    oracle on the same allocation, and the next allocation is the rule
    applied to the GPU's variances, exactly."""
    s = oracle.plus_nstrat(2, 4000)
    nh = s * s
    counts = np.full(nh, 2, np.int32)
    counts[::97] += 1
    counts[300] = 2500
    assert counts.sum() <= 4000 + 2 * nh and counts[:300].sum() < 1024 < counts[:301].sum() - 2048
    g = v.Vegas(2, 20, 3)
    try:
        g.strat_set(4000, counts)
        g.set(v.VEGAS_OPT_STRAT, 1)
        I, e, c, per, _ = g.iterate(4000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)
        ref = oracle.iterate_plus(2, 20, 3, 4000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS, alloc=counts)
        per_agrees(per, ref, counts)
        _, alloc2, var = g.strat()
        var_agrees(var, ref, counts)
        assert np.array_equal(alloc2, oracle.plus_allocate(4000, var))
    finally:
        g.close()


def test_plus_reduces_the_variance_on_the_gpu():
    iid, params, ndim, nbins = CASES["gauss_d2"]
    errs = []
    for strat in (0, 1):
        g = v.Vegas(ndim, nbins, 5)
        try:
            g.set(v.VEGAS_OPT_STRAT, strat)
            g.iterate(200_000, 4, iid, params)
            I, e, c, per, _ = g.iterate(200_000, 5, iid, params)
            errs.append(e)
        finally:
            g.close()
    assert errs[1] * 3 < errs[0]


@pytest.mark.parametrize("name", ["dy", "ee3j"])
def test_plus_fp32_form_against_oracle(name):
    iid, params, ndim, nbins = CASES[name]
    g = gpu_state(iid, params, ndim, nbins, 100_000, 2, precision="fp32")
    try:
        edges = g.grid
        s, alloc, _ = g.strat()
        I, e, c, per, _ = g.iterate(100_000, 1, iid, params)
    finally:
        g.close()
    ref = oracle.iterate_plus(ndim, nbins, 1234, 100_000, 1, iid, params, edges=edges, alloc=alloc,
                              iteration=2)
    assert rel(per[:, 0], ref.per_iter[:, 0]) < 2e-5
    assert rel(per[:, 1], ref.per_iter[:, 1]) < 2e-4


@pytest.mark.parametrize("ndim,ncall", [(1, 2 ** 20), (16, 300_000), (1, 8), (3, 10)])
def test_plus_extreme_shapes_match_oracle(ndim, ncall):
    """One axis with a quarter of a million strata, sixteen axes, and the
    smallest call counts: a stage from the uniform start, then one iteration
    from the GPU's state, against the oracle."""
    iid, params = v.VEGAS_GAUSS, GAUSS_PARAMS
    nbins = 20
    g = gpu_state(iid, params, ndim, nbins, ncall, 2)
    try:
        edges = g.grid
        s, alloc, _ = g.strat()
        I, e, c, per, _ = g.iterate(ncall, 1, iid, params)
        s2, alloc2, var = g.strat()
    finally:
        g.close()
    ref = oracle.iterate_plus(ndim, nbins, 1234, ncall, 1, iid, params, edges=edges, alloc=alloc,
                              iteration=2)
    assert s == ref.nstrat and len(alloc) == s ** ndim
    per_agrees(per, ref, alloc)
    var_agrees(var, ref, alloc)
    assert np.array_equal(alloc2, oracle.plus_allocate(ncall, var))


@pytest.mark.parametrize("beta", [0.0, 0.25, 0.5, 1.0])
def test_plus_damping_values_match_oracle(beta):
    iid, params, ndim, nbins = CASES["dy"]
    g = gpu_state(iid, params, ndim, nbins, 20_000, 2, beta=beta)
    try:
        edges = g.grid
        s, alloc, _ = g.strat()
        I, e, c, per, _ = g.iterate(20_000, 1, iid, params)
        s2, alloc2, var = g.strat()
    finally:
        g.close()
    ref = oracle.iterate_plus(ndim, nbins, 1234, 20_000, 1, iid, params, edges=edges, alloc=alloc,
                              iteration=2, beta=beta)
    per_agrees(per, ref, alloc)
    var_agrees(var, ref, alloc)
    assert np.array_equal(alloc2, oracle.plus_allocate(20_000, var, beta=beta))
    if beta == 0.0:  # every hypercube weighs the same: the allocation stays uniform
        assert np.all(alloc2 == 20_000 // len(alloc2))


def test_plus_checkpoint_with_saved_allocation_continues_bit_exactly():
    """A checkpoint plus the allocation saved beside it (vegas_strat_get /
    vegas_strat_set) continue a VEGAS+ run bit for bit in a new context."""
    iid, params, ndim, nbins = CASES["dy"]
    a = gpu_state(iid, params, ndim, nbins, 20_000, 2)
    try:
        blob = a.state()
        s, alloc, _ = a.strat()
        ref = a.iterate(20_000, 2, iid, params)
        ref_grid = a.grid
    finally:
        a.close()
    b = v.Vegas(ndim, nbins, 99)
    try:
        b.restore(blob)
        b.set(v.VEGAS_OPT_STRAT, 1)
        b.strat_set(20_000, alloc)
        got = b.iterate(20_000, 2, iid, params)
        assert np.array_equal(got[3], ref[3]) and got[:3] == ref[:3]
        assert np.array_equal(b.grid, ref_grid)
    finally:
        b.close()
