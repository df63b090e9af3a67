"""GPU histograms of the observable against the oracle, through the C ABI.

The per-bin sums of w and w^2 are exact integer sums rounded once, so the
FP64 form matches the oracle to 1e-12 on the same grid and is bit-identical
for every launch shape; the stage's histogram adds up to its integral.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import (DY_PARAMS, DYNLO_PARAMS, EE3J_PARAMS, GAUSS_PARAMS,
                                              GAUSS_SHIFTED_PARAMS)

pytestmark = pytest.mark.gpu

# name: (integrand, params, ndim, nbins, histogram (nh, lo, hi))
CASES = {
    "gauss": (v.VEGAS_GAUSS, GAUSS_PARAMS, 4, 50, (20, 0.2, 0.8)),
    "gauss_signed": (v.VEGAS_GAUSS, GAUSS_SHIFTED_PARAMS, 2, 50, (16, 0.0, 1.0)),
    "dy": (v.VEGAS_DY, DY_PARAMS, 4, 100, (60, 60.0, 120.0)),
    "ee3j": (v.VEGAS_EE3J, EE3J_PARAMS, 5, 100, (30, 2 / 3, 1.0)),
    "dy_nlo": (v.VEGAS_DY_NLO, DYNLO_PARAMS, 13, 50, (12, 66.0, 114.0)),
}


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def close_with_zeros(got, want, tol):
    """Same zero pattern, and the nonzero entries within tol relative."""
    got, want = np.asarray(got), np.asarray(want)
    assert np.array_equal(got == 0, want == 0)
    nz = want != 0
    if np.any(nz):
        assert rel(got[nz], want[nz]) < tol


def gpu_stage(iid, params, ndim, nbins, hist, ncall, itmx, *, warm=2, adapt=0, precision="fp64",
              **opts):
    """A warm-up stage (no histogram), then a stage with the histogram on the
    grid it left (frozen unless adapt)."""
    g = v.Vegas(ndim, nbins, 1234, precision=precision)
    try:
        for k, val in opts.items():
            g.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
        g.iterate(max(ncall // 2, 2), warm, iid, params)
        edges = g.grid
        g.set(v.VEGAS_OPT_ADAPT, adapt)
        g.hist_set(*hist)
        I, e, c, per, _ = g.iterate(ncall, itmx, iid, params)
        val, err, last = g.hist()
        return dict(edges=edges, integral=I, error=e, per_iter=per, value=val, err=err, last=last,
                    grid=g.grid, sums=g.last_sums())
    finally:
        g.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ncall", [20 * 1024 + 37, 1500])
def test_hist_fp64_matches_oracle(name, ncall):
    iid, params, ndim, nbins, hist = CASES[name]
    itmx = 3
    gpu = gpu_stage(iid, params, ndim, nbins, hist, ncall, itmx)
    ref = oracle.iterate(ndim, nbins, 1234, ncall, itmx, iid, params, edges=gpu["edges"],
                         iteration=2, adapt=False, want_sums=True, hist=hist)
    assert rel(gpu["per_iter"], ref.per_iter) < 1e-12
    close_with_zeros(gpu["last"][0], ref.hist_last[0], 1e-12)
    close_with_zeros(gpu["last"][1], ref.hist_last[1], 1e-12)
    close_with_zeros(gpu["value"], ref.hist_value, 1e-12)
    close_with_zeros(gpu["err"], ref.hist_error, 1e-11)
    # the bins add up to the integral, the last sums to its sum w, sum w^2
    assert abs(np.sum(gpu["value"]) - gpu["integral"]) <= 1e-12 * abs(gpu["integral"])
    assert abs(np.sum(gpu["last"][0]) - gpu["sums"][0]) <= 1e-12 * abs(gpu["sums"][0])
    assert abs(np.sum(gpu["last"][1]) - gpu["sums"][1]) <= 1e-12 * gpu["sums"][1]


def test_signed_weights_reach_negative_bins():
    iid, params, ndim, nbins, hist = CASES["gauss_signed"]
    gpu = gpu_stage(iid, params, ndim, nbins, hist, 50_000, 3)
    assert gpu["integral"] < 0
    assert np.any(gpu["value"] < 0) and np.any(gpu["value"] > 0)
    assert np.any(gpu["last"][0] < 0)


@pytest.mark.parametrize("name", ["dy", "ee3j", "gauss_signed"])
def test_hist_bit_identical_across_launch_shapes(name):
    """Graph or plain launches, with and without PDL chaining: the same bits."""
    iid, params, ndim, nbins, hist = CASES[name]
    outs = [gpu_stage(iid, params, ndim, nbins, hist, 9 * 1024 + 5, 3, adapt=1, graph=gr, pdl=pd)
            for gr in (1, 0) for pd in (1, 0)]
    for o in outs[1:]:
        for key in ("value", "err", "last", "per_iter", "grid"):
            assert np.array_equal(o[key], outs[0][key]), key


def test_hist_leaves_the_integration_unchanged():
    """The same stage with and without a histogram: the same iterations, grid
    and sums, bit for bit (the histogram only adds slots)."""
    iid, params, ndim, nbins, hist = CASES["dy"]
    res = []
    for h in (hist, None):
        g = v.Vegas(ndim, nbins, 77)
        try:
            if h:
                g.hist_set(*h)
            I, e, c, per, _ = g.iterate(30_000, 3, iid, params)
            res.append((per, g.grid, g.last_sums()))
        finally:
            g.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_hist_adapting_stage_adds_up():
    """With the grid adapting inside the stage, the stage's histogram still
    adds up to its integral, and each bin's error is finite and positive
    where the bin has events."""
    iid, params, ndim, nbins, hist = CASES["dy"]
    gpu = gpu_stage(iid, params, ndim, nbins, hist, 100_000, 5, adapt=1)
    assert abs(np.sum(gpu["value"]) - gpu["integral"]) <= 1e-12 * abs(gpu["integral"])
    inner = slice(1, hist[0] + 1)
    assert np.all(gpu["value"][inner] > 0) and np.all(gpu["err"][inner] > 0)
    assert gpu["value"][0] == 0 and gpu["value"][-1] == 0  # m_ll is generated in [60, 120]


@pytest.mark.parametrize("name", ["dy", "ee3j", "dy_nlo"])
def test_hist_fp32_form_against_oracle(name):
    """The FP32 integrand form, observable and bin decision in FP32: bins with
    a visible share agree with the FP64 oracle to the FP32 form's accuracy."""
    iid, params, ndim, nbins, hist = CASES[name]
    gpu = gpu_stage(iid, params, ndim, nbins, hist, 200_000, 3, precision="fp32")
    ref = oracle.iterate(ndim, nbins, 1234, 200_000, 3, iid, params, edges=gpu["edges"],
                         iteration=2, adapt=False, hist=hist)
    big = np.abs(ref.hist_value) > 0.01 * np.max(np.abs(ref.hist_value))
    # an FP32 m_ll is off by ~5e-5 GeV, so a few events per edge change bin
    assert rel(gpu["value"][big], ref.hist_value[big]) < 1e-3
    assert abs(np.sum(gpu["value"]) - gpu["integral"]) <= 1e-12 * abs(gpu["integral"])


def test_hist_set_validation_and_off():
    g = v.Vegas(4, 20, 1)
    try:
        for bad in [(-1, 0.0, 1.0), (v.VEGAS_HIST_MAX_BINS + 1, 0.0, 1.0), (10, 1.0, 1.0),
                    (10, 2.0, 1.0), (10, float("nan"), 1.0), (10, 0.0, float("inf"))]:
            with pytest.raises(v.VegasError):
                g.hist_set(*bad)
        with pytest.raises(v.VegasError):  # nothing filled yet
            g.hist()
        g.hist_set(10, 0.0, 1.0)
        with pytest.raises(v.VegasError):  # set, but no stage has filled it
            g.hist()
        g.iterate(5000, 2, v.VEGAS_GAUSS, GAUSS_PARAMS)
        val, err, last = g.hist()
        assert val.shape == (12,) and last.shape == (2, 12)
        g.hist_set(0)
        with pytest.raises(v.VegasError):
            g.hist()
        g.iterate(5000, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)  # runs without a histogram
    finally:
        g.close()


@pytest.mark.parametrize("hist", [(1, 0.0, 1.0), (v.VEGAS_HIST_MAX_BINS, 0.0, 1.0),
                                  (10, 2.0, 3.0), (10, -3.0, -2.0)])
def test_hist_edge_binnings_match_oracle(hist):
    """One bin, the most bins, and ranges no event reaches (everything in the
    underflow, or in the overflow): the FP64 form against the oracle."""
    iid, params, ndim, nbins, _ = CASES["gauss"]
    gpu = gpu_stage(iid, params, ndim, nbins, hist, 20 * 1024 + 37, 2)
    ref = oracle.iterate(ndim, nbins, 1234, 20 * 1024 + 37, 2, iid, params, edges=gpu["edges"],
                         iteration=2, adapt=False, want_sums=True, hist=hist)
    close_with_zeros(gpu["last"][0], ref.hist_last[0], 1e-12)
    close_with_zeros(gpu["last"][1], ref.hist_last[1], 1e-12)
    close_with_zeros(gpu["value"], ref.hist_value, 1e-12)
    close_with_zeros(gpu["err"], ref.hist_error, 1e-11)
    if hist[1] >= 1.0:  # x_0 < 1 <= lo: everything is underflow
        assert np.count_nonzero(gpu["value"]) == 1 and gpu["value"][0] != 0
    if hist[2] <= 0.0:  # hi <= 0 < x_0: everything is overflow
        assert np.count_nonzero(gpu["value"]) == 1 and gpu["value"][-1] != 0
