"""Batched form: many integrations of uneven dimension, call count and
integrand advanced by persistent fill launches, one per iteration, dimension
class and integrand (requires a GB300).

Bar: every member bit-identical to a single context with the same Philox
batch word (any schedule, any events-per-thread, graph or not); FP64 members
within 1e-12 relative of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import DY_PARAMS, EE3J_PARAMS, GAUSS_PARAMS

pytestmark = pytest.mark.gpu

NBINS = 50
SEED = 4321
# (ndim, ncall, integrand, params): uneven sizes, ragged tails, every integrand
# in every dimension class it can take (4, 8, 16 axes): all eight work lists
MEMBERS = [
    (2, 5_000, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (4, 20_011, v.VEGAS_DY, DY_PARAMS),
    (5, 9_000, v.VEGAS_EE3J, EE3J_PARAMS),
    (8, 3_001, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (6, 1_500, v.VEGAS_DY, DY_PARAMS),
    (16, 2_500, v.VEGAS_GAUSS, GAUSS_PARAMS),
    (12, 2_047, v.VEGAS_DY, DY_PARAMS),
    (10, 3_333, v.VEGAS_EE3J, EE3J_PARAMS),
]
STAGES = (3, 2)


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def run_batch(precision="fp64", **opts):
    B = v.VegasBatch(MEMBERS, NBINS, SEED, precision=precision)
    try:
        for k, val in opts.items():
            B.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
        out = [B.iterate(itmx) for itmx in STAGES]
        grids = [B.grid(b) for b in range(len(MEMBERS))]
    finally:
        B.close()
    return out, grids


def run_single(b, precision="fp64"):
    d, ncall, iid, params = MEMBERS[b]
    g = v.Vegas(d, NBINS, SEED, precision=precision)
    try:
        g.set(v.VEGAS_OPT_BATCH_ID, b)
        out = [g.iterate(ncall, itmx, iid, params)[:4] for itmx in STAGES]
        return out, g.grid
    finally:
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_bit_identical_to_single_contexts(precision):
    out, grids = run_batch(precision)
    for b in range(len(MEMBERS)):
        single, grid = run_single(b, precision)
        for s, (I, e, c, per) in enumerate(single):
            bI, be, bc, bper = (x[b] for x in out[s])
            assert bI == I and be == e and bc == c, (b, s)
            assert np.array_equal(bper, per), (b, s)
        assert np.array_equal(grids[b], grid), b


def test_batch_launch_shapes_bit_identical():
    base, bgrids = run_batch(ept=4)
    for opts in ({"ept": 8}, {"ept": 4, "graph": 0}, {"ept": 4, "batch_grid": 4},
                 {"ept": 8, "batch_grid": 3}):
        out, grids = run_batch(**opts)
        for s in range(len(STAGES)):
            for a, b in zip(out[s], base[s]):
                assert np.array_equal(a, b), opts
        for a, b in zip(grids, bgrids):
            assert np.array_equal(a, b), opts


def test_batch_fp64_matches_oracle():
    """Every member, iteration by iteration, against the oracle started from
    the member's grid (one-iteration stages; the sparse peaked members shrink
    bins enough that a chain of refinements magnifies last-bit differences)."""
    n = len(MEMBERS)
    B = v.VegasBatch(MEMBERS, NBINS, SEED)
    try:
        grids = [[B.grid(b) for b in range(n)]]
        outs = []
        for _ in range(3):
            outs.append(B.iterate(1))
            grids.append([B.grid(b) for b in range(n)])
    finally:
        B.close()
    for b, (d, ncall, iid, params) in enumerate(MEMBERS):
        for k in range(3):
            ref = oracle.iterate(d, NBINS, SEED, ncall, 1, iid, params, edges=grids[k][b],
                                 iteration=k, batch=b)
            I, e, c, per = (x[b] for x in outs[k])
            assert rel(per, ref.per_iter) < 1e-12, (b, k)
            assert rel(I, ref.integral) < 1e-12 and rel(e, ref.error) < 1e-12, (b, k)
            assert np.max(np.abs(grids[k + 1][b] - ref.edges)) <= 1e-12, (b, k)


def test_batch_without_adaptation_keeps_uniform_grid():
    out, grids = run_batch(adapt=0)
    for b, (d, _, _, _) in enumerate(MEMBERS):
        assert np.array_equal(grids[b], oracle.uniform_edges(d, NBINS))


def test_batch_invalid_arguments():
    with pytest.raises(v.VegasError):
        v.VegasBatch([(3, 1000, v.VEGAS_DY, DY_PARAMS)], NBINS)  # DY needs ndim >= 4
    with pytest.raises(v.VegasError):
        v.VegasBatch([(2, 1, v.VEGAS_GAUSS, GAUSS_PARAMS)], NBINS)  # ncall < 2
    with pytest.raises(v.VegasError):
        v.VegasBatch([(17, 1000, v.VEGAS_GAUSS, GAUSS_PARAMS)], NBINS)
    with pytest.raises(v.VegasError):
        v.VegasBatch([(2, 1000, v.VEGAS_GAUSS, (-1.0,))], NBINS)
    B = v.VegasBatch([(2, 1000, v.VEGAS_GAUSS, GAUSS_PARAMS)], NBINS)
    try:
        with pytest.raises(v.VegasError):
            B.set(v.VEGAS_OPT_PRECISION, 1)
        with pytest.raises(v.VegasError):
            B.set(v.VEGAS_OPT_EPT, 2)
        with pytest.raises(v.VegasError):
            v.vegas_batch_grid_get(B.h, 1, 2, NBINS)
    finally:
        B.close()
