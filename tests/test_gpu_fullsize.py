"""GPU path vs the oracle at the sizes the benchmark runs (requires a GB300).

The Drell-Yan workload of the benchmark (d = 4, N = 100, 10 iterations x 1e6
calls; 977 tiles, which the single-level reduce reads with one 256-thread
group per slot, four tiles per thread, from registers) and the other
workloads at their full sizes: the Gaussian (5 x 1e5), the 3-jet form (1e7
calls per iteration: 9,766 tiles, 38 per thread, read in two passes), the
Drell-Yan gradient (1e8 calls per iteration, the two-level reduce) and the
batch of 64 integrations.  Sections 2.1 and 2.2: the same events give the same result
whatever the split of the work.

Bar (FP64 form): each iteration, run by the oracle from the GPU's grid and
iteration counter, gives I_k and sigma_k within 1e-12 relative, the refined
edges within 1e-12 absolute and the iteration's sums within 1e-12 relative
with the same zero pattern.  A multi-iteration stage on the GPU gives the
same bits as the chain of one-iteration stages, and every launch shape
(events per thread, CUDA graph, programmatic dependent launch) gives the same
bits.  FP32 form: each I_k within 2e-5 and sigma_k within 2e-4 of the FP64
oracle on the same events and grid (the achieved errors are printed).
"""
import numpy as np
import pytest

import oracle
from paper_1503_06182_gb300 import vegas as v
from paper_1503_06182_gb300.workloads import DY_PARAMS, EE3J_PARAMS, GAUSS_PARAMS, batch_spec

pytestmark = pytest.mark.gpu

SEED = 1234
DY_SHAPE = (4, 100, 1_000_000, 10)  # ndim, nbins, calls per iteration, iterations


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def chain(ndim, nbins, ncall, itmx, iid, params, precision="fp64", **opts):
    """itmx one-iteration stages on one context: the grid before each
    iteration, the per-iteration records and each iteration's sums."""
    g = v.Vegas(ndim, nbins, SEED, precision=precision)
    try:
        for k, val in opts.items():
            g.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
        grids, per, sums = [g.grid], [], []
        for _ in range(itmx):
            per.append(g.iterate(ncall, 1, iid, params)[3][0])
            sums.append(g.last_sums())
            grids.append(g.grid)
        return grids, np.array(per), sums
    finally:
        g.close()


def stage(ndim, nbins, ncall, itmx, iid, params, precision="fp64", **opts):
    """One stage of itmx iterations (one call, as the benchmark runs it)."""
    g = v.Vegas(ndim, nbins, SEED, precision=precision)
    try:
        for k, val in opts.items():
            g.set(getattr(v, "VEGAS_OPT_" + k.upper()), val)
        I, e, c, per, _ = g.iterate(ncall, itmx, iid, params)
        return dict(integral=I, error=e, chi2=c, per_iter=per, edges=g.grid, sums=g.last_sums())
    finally:
        g.close()


def check_iterations_fp64(ndim, nbins, ncall, iid, params, grids, per, sums):
    """Each GPU iteration against the oracle restarted from the GPU's grid."""
    for k in range(len(per)):
        ref = oracle.iterate(ndim, nbins, SEED, ncall, 1, iid, params, edges=grids[k],
                             iteration=k, want_sums=True)
        assert rel(per[k], ref.per_iter[0]) < 1e-12, (k, per[k], ref.per_iter[0])
        assert np.max(np.abs(grids[k + 1] - ref.edges)) < 1e-12, k
        s, sr = sums[k], ref.sums
        assert rel(s[:2], sr[:2]) < 1e-12, k
        nz = sr[2:] != 0
        assert np.array_equal(s[2:] != 0, nz), k
        assert rel(s[2:][nz], sr[2:][nz]) < 1e-12, k


def check_iterations_fp32(name, ndim, nbins, ncall, iid, params, grids, per):
    """FP32-integrand iterations against the FP64 oracle on the same grid."""
    eI = eS = 0.0
    for k in range(len(per)):
        ref = oracle.iterate(ndim, nbins, SEED, ncall, 1, iid, params, edges=grids[k],
                             iteration=k)
        eI = max(eI, rel(per[k][0], ref.per_iter[0, 0]))
        eS = max(eS, rel(per[k][1], ref.per_iter[0, 1]))
    print(f"{name}: FP32 form vs FP64 oracle over {len(per)} iterations x {ncall} calls: "
          f"max rel err I_k {eI:.2e}, sigma_k {eS:.2e}")
    assert eI < 2e-5
    assert eS < 2e-4


# ------------------------------------------------------ the benchmark's workload
@pytest.fixture(scope="module")
def dy_fp64():
    ndim, nbins, ncall, itmx = DY_SHAPE
    return chain(ndim, nbins, ncall, itmx, v.VEGAS_DY, DY_PARAMS)


@pytest.fixture(scope="module")
def dy_fp32():
    ndim, nbins, ncall, itmx = DY_SHAPE
    return chain(ndim, nbins, ncall, itmx, v.VEGAS_DY, DY_PARAMS, precision="fp32")


def test_bench_workload_fp64_iterations_match_oracle(dy_fp64):
    ndim, nbins, ncall, _ = DY_SHAPE
    grids, per, sums = dy_fp64
    check_iterations_fp64(ndim, nbins, ncall, v.VEGAS_DY, DY_PARAMS, grids, per, sums)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bench_stage_equals_chain_of_iterations(precision, dy_fp64, dy_fp32):
    """The 10-iteration stage (one CUDA graph, programmatically chained
    kernels, autotuned events per thread) gives the bits of the chain of
    one-iteration stages; its combination is the oracle's combination of
    those iterations."""
    grids, per, sums = dy_fp64 if precision == "fp64" else dy_fp32
    out = stage(*DY_SHAPE, v.VEGAS_DY, DY_PARAMS, precision=precision)
    assert np.array_equal(out["per_iter"], per)
    assert np.array_equal(out["edges"], grids[-1])
    assert np.array_equal(out["sums"], sums[-1])
    I, e, c = oracle.combine(per[:, 0], per[:, 1])
    assert rel(out["integral"], I) < 1e-13
    assert rel(out["error"], e) < 1e-13
    assert abs(out["chi2"] - c) < 1e-10 * max(1.0, c)


def test_bench_workload_fp32_error_vs_oracle(dy_fp32):
    ndim, nbins, ncall, _ = DY_SHAPE
    grids, per, _ = dy_fp32
    check_iterations_fp32("drell_yan d4 N100 1e6", ndim, nbins, ncall, v.VEGAS_DY, DY_PARAMS,
                          grids, per)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bench_workload_launch_shapes_bit_identical(precision):
    """Events per thread 1/2/4/8, CUDA graph on/off, programmatic dependent
    launch on/off: the same bits for the 10 x 1e6 stage."""
    shapes = [(ept, graph, pdl) for ept in (1, 2, 4, 8) for graph in (1, 0) for pdl in (1, 0)]
    if precision == "fp64":
        shapes = [s for s in shapes if s[2] == 1 or s[0] == 4]
    outs = [stage(*DY_SHAPE, v.VEGAS_DY, DY_PARAMS, precision=precision, ept=ept, graph=graph,
                  pdl=pdl) for ept, graph, pdl in shapes]
    for s, o in zip(shapes[1:], outs[1:]):
        assert np.array_equal(o["per_iter"], outs[0]["per_iter"]), s
        assert np.array_equal(o["edges"], outs[0]["edges"]), s
        assert np.array_equal(o["sums"], outs[0]["sums"]), s
        assert (o["integral"], o["error"], o["chi2"]) == \
            (outs[0]["integral"], outs[0]["error"], outs[0]["chi2"]), s


# ------------------------------------------------------------- other workloads
def test_gauss_workload_fp64_matches_oracle():
    """The Gaussian, d = 4, N = 50, 5 x 1e5 (FP64): every iteration from the
    GPU's grid, and the stage against the stage's combination."""
    ndim, nbins, ncall, itmx = 4, 50, 100_000, 5
    grids, per, sums = chain(ndim, nbins, ncall, itmx, v.VEGAS_GAUSS, GAUSS_PARAMS)
    check_iterations_fp64(ndim, nbins, ncall, v.VEGAS_GAUSS, GAUSS_PARAMS, grids, per, sums)
    out = stage(ndim, nbins, ncall, itmx, v.VEGAS_GAUSS, GAUSS_PARAMS)
    assert np.array_equal(out["per_iter"], per)
    assert np.array_equal(out["edges"], grids[-1])


def test_ee3j_1e7_calls_fp64_matches_oracle():
    """3-jet form, d = 5, N = 100, 1e7 calls per iteration (the reduce's
    two-pass path: more tiles than a group holds in registers), two
    iterations from the GPU's grids."""
    ndim, nbins, ncall = 5, 100, 10_000_000
    grids, per, sums = chain(ndim, nbins, ncall, 2, v.VEGAS_EE3J, EE3J_PARAMS)
    check_iterations_fp64(ndim, nbins, ncall, v.VEGAS_EE3J, EE3J_PARAMS, grids, per, sums)


def test_ee3j_workload_fp32_full_stage():
    """The 3-jet workload as the benchmark runs it (FP32, 10 x 1e7): the
    stage equals the chain of iterations, every iteration is within the FP32
    bar of the oracle, and events per thread 2 and 4 give the same bits."""
    ndim, nbins, ncall, itmx = 5, 100, 10_000_000, 10
    grids, per, _ = chain(ndim, nbins, ncall, itmx, v.VEGAS_EE3J, EE3J_PARAMS, precision="fp32")
    check_iterations_fp32("ee3j d5 N100 1e7", ndim, nbins, ncall, v.VEGAS_EE3J, EE3J_PARAMS,
                          grids, per)
    outs = [stage(ndim, nbins, ncall, itmx, v.VEGAS_EE3J, EE3J_PARAMS, precision="fp32", ept=e)
            for e in (4, 2)]
    for o in outs:
        assert np.array_equal(o["per_iter"], per)
        assert np.array_equal(o["edges"], grids[-1])


def test_gradient_1e8_calls_matches_oracle():
    """The Drell-Yan gradient at the workload's 1e8 calls per iteration, on a
    grid adapted by a forward warm-up: FP64 against the oracle (1e-10 of
    |G| + sigma_G, as the smaller cases), FP32 within 1e-4 of it, and the
    FP32 form's bits the same for 1, 2 and 4 events per thread."""
    ndim, nbins, ncall = 4, 100, 100_000_000
    res = {}
    for prec in ("fp64", "fp32"):
        g = v.Vegas(ndim, nbins, SEED, precision=prec)
        try:
            g.iterate(1_000_000, 3, v.VEGAS_DY, DY_PARAMS)
            g.set(v.VEGAS_OPT_ADAPT, 0)
            edges = g.grid
            st = g.state()
            res[prec] = g.adjoint(ncall, 1, DY_PARAMS)
            if prec == "fp32":
                for ept in (1, 2, 4):
                    g.restore(st)
                    g.set(v.VEGAS_OPT_EPT, ept)
                    o = g.adjoint(ncall, 1, DY_PARAMS)
                    for a, b in zip(o, res[prec]):
                        assert np.array_equal(np.asarray(a), np.asarray(b)), ept
        finally:
            g.close()
        if prec == "fp64":
            ref = oracle.adjoint(ndim, nbins, SEED, ncall, 1, DY_PARAMS, edges=edges, iteration=3)
    grad, gerr, I, e, _ = res["fp64"]
    assert np.all(np.abs(grad - ref.grad) <= 1e-10 * (np.abs(ref.grad) + ref.grad_err))
    assert np.all(np.abs(gerr - ref.grad_err) <= 1e-9 * ref.grad_err)
    assert rel(I, ref.integral) < 1e-12
    g32 = res["fp32"][0]
    err = np.abs(g32 - ref.grad) / (np.abs(ref.grad) + ref.grad_err)
    print("gradient 1e8 calls: FP32 form max |dG|/(|G|+sigma_G) =", err.max())
    assert err.max() < 1e-4


def test_batch64_workload_matches_oracle_and_single_contexts():
    """The 64-integration workload (spec from seed 1234): one FP64 iteration
    of every member against the oracle, and the FP32 members of a
    10-iteration batched stage bit-identical to single contexts."""
    spec = batch_spec(64, SEED)
    members = [(m.ndim, m.ncall, m.integrand, m.params) for m in spec]
    nbins = 100
    B = v.VegasBatch(members, nbins, SEED)
    try:
        grids = [B.grid(b) for b in range(len(members))]
        I, e, c, per = B.iterate(1)
        after = [B.grid(b) for b in range(len(members))]
    finally:
        B.close()
    for b, (d, ncall, iid, params) in enumerate(members):
        ref = oracle.iterate(d, nbins, SEED, ncall, 1, iid, params, edges=grids[b], iteration=0,
                             batch=b)
        assert rel(per[b], ref.per_iter) < 1e-12, b
        assert np.max(np.abs(after[b] - ref.edges)) < 1e-12, b
    B = v.VegasBatch(members, nbins, SEED, precision="fp32")
    try:
        out = B.iterate(10)
        bgrids = [B.grid(b) for b in range(len(members))]
    finally:
        B.close()
    for b, (d, ncall, iid, params) in enumerate(members):
        g = v.Vegas(d, nbins, SEED, precision="fp32")
        try:
            g.set(v.VEGAS_OPT_BATCH_ID, b)
            sI, se, sc, sper, _ = g.iterate(ncall, 10, iid, params)
            assert np.array_equal(sper, out[3][b]), b
            assert (sI, se, sc) == (out[0][b], out[1][b], out[2][b]), b
            assert np.array_equal(g.grid, bgrids[b]), b
        finally:
            g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_shaped_gauss13_iterations_match_oracle(precision):
    """The paper's run shape on the 13-axis Gaussian (Section 3.2: 1e4 events per
    production iteration): each iteration against the oracle from the GPU's grid
    and counter.  At so few events per iteration VEGAS itself is unreliable in 13
    dimensions (single iterations scatter by factors of several), so the FP32 and
    FP64 chains part; each step still agrees."""
    ndim, nbins, ncall = 13, 50, 10_000
    grids, per, sums = chain(ndim, nbins, ncall, 6, v.VEGAS_GAUSS, GAUSS_PARAMS,
                             precision=precision)
    if precision == "fp64":
        check_iterations_fp64(ndim, nbins, ncall, v.VEGAS_GAUSS, GAUSS_PARAMS, grids, per, sums)
    else:
        check_iterations_fp32("gauss d13 N50 1e4", ndim, nbins, ncall, v.VEGAS_GAUSS,
                              GAUSS_PARAMS, grids, per)
